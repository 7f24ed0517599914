// Subpixel blend WITHOUT view-coherent remapping: the ablation of Sec. 4.3
// ("Ours w/o remap" in the ablation study, T3). Threads take the tile's
// subpixels in plain row-major order, so neighbouring threads usually belong
// to different views and clusters; each thread finds its own list
// [S_tk, E_tk) through its view index (Alg. 2 Alpha-Blend with Psi the
// identity) and walks it straight from global memory. The per-entry
// arithmetic is the remapped kernel's, so the image is the same; only the
// memory access pattern differs.
#include "lfd_internal.h"

namespace lfd {
namespace {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;

template <bool COUNT>
__global__ void __launch_bounds__(256) k_blend_raster(PanelGeom g, BlendArgs a) {
  if (a.P_dev && *a.P_dev > a.P_cap) return;  // capacity overflow: leave the image
  const int t = blockIdx.x;
  const int tx = t % g.TX, ty = t / g.TX;
  const int w = min(g.TW, g.W - tx * g.TW);
  const int h = min(g.TH, g.H - ty * g.TH);
  const int n = 3 * w * h;
  unsigned long long n_walk = 0;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const int u = r % 3;
    const int xl = (r / 3) % w;
    const int yl = (r / 3) / w;
    const int x = tx * g.TW + xl, y = ty * g.TH + yl;
    const int64_t oidx = ((int64_t)y * g.W + x) * 3 + u;
    const int view = a.V[oidx];
    const int k = view / g.C;
    const int slot = view - k * g.C;
    const uint2 rg = a.ranges[(size_t)t * g.K + k];
    const float px = (float)x + 0.5f, py = (float)y + 0.5f;
    float T = 1.f, acc = 0.f;
    for (uint32_t e = rg.x; e < rg.y; ++e) {
      if (COUNT) ++n_walk;
      const size_t rec = (size_t)k * a.M + a.list[e];
      const float4 c4 = reinterpret_cast<const float4*>(a.conic_opacity)[rec];
      const float4 co = make_float4(-0.5f * kLog2e * c4.x, -kLog2e * c4.y, -0.5f * kLog2e * c4.z, c4.w);
      const float2 mu = reinterpret_cast<const float2*>(a.means2d)[rec * g.C + slot];
      const float dx = px - mu.x;
      const float dy = py - mu.y;
      const float power = quad_power(co.x, co.y, co.z, dx, dy);
      if (power > 0.f) continue;
      const float v = co.w * ex2_approx(power);
      if (!(v >= kAlphaMin)) continue;
      const float alpha = fminf(kAlphaMax, v);
      const float Tn = T * (1.f - alpha);
      if (Tn < kTMin) break;
      const float4 cl = reinterpret_cast<const float4*>(a.color_tau)[rec];
      const float c = u == 0 ? cl.x : (u == 1 ? cl.y : cl.z);
      acc += c * alpha * T;
      T = Tn;
    }
    const float bg = u == 0 ? a.bg[0] : (u == 1 ? a.bg[1] : a.bg[2]);
    a.out[oidx] = acc + T * bg;
  }
  if (COUNT) {
    unsigned long long c = n_walk;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) {
      atomicAdd(a.eval_counter, c);
      atomicAdd(a.eval_counter + 1, c);
    }
  }
}

}  // namespace

cudaError_t launch_blend_raster(const PanelGeom& g, const BlendArgs& a, cudaStream_t s) {
  if (g.T == 0) return cudaSuccess;
  const int block = min(256, ((g.cap + 31) / 32) * 32);
  if (a.eval_counter)
    k_blend_raster<true><<<g.T, block, 0, s>>>(g, a);
  else
    k_blend_raster<false><<<g.T, block, 0, s>>>(g, a);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace lfd
