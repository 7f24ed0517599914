// Full-frame baseline (Sec. 1 and Sec. 5.1: "render all multi-view images at
// full resolution before interlacing"; the "3DGS" rows of T1/T2): every view
// is rasterised as an ordinary 3DGS image with its own lists (one view per
// cluster, no attribute reuse), one thread per pixel blending all three
// channels with one alpha per Gaussian; the interlacing is fused into the
// write: a pixel of view j stores only the channels (x, y, u) whose view index
// is j. The pixels of every view are still all computed, which is the work
// the subpixel method avoids.
#include "lfd_internal.h"

namespace lfd {
namespace {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;

// Grid: (view j, tile t), view-major; clusters are single views (C = 1).
template <bool COUNT>
__global__ void __launch_bounds__(512) k_blend_fullframe(PanelGeom g, BlendArgs a) {
  if (a.P_dev && *a.P_dev > a.P_cap) return;  // capacity overflow: leave the image
  extern __shared__ float4 smem[];
  const int NB = blockDim.x;
  float4* s_co = smem;
  float4* s_col = smem + NB;
  float2* s_mean = reinterpret_cast<float2*>(smem + 2 * NB);
  const int j = blockIdx.x / g.T;
  const int t = blockIdx.x - j * g.T;
  const int tx = t % g.TX, ty = t / g.TX;
  const int xl = threadIdx.x % g.TW, yl = threadIdx.x / g.TW;
  const int x = tx * g.TW + xl, y = ty * g.TH + yl;
  const bool inside = yl < g.TH && x < g.W && y < g.H;
  const uint2 rg = a.ranges[(size_t)t * g.K + j];
  const float px = (float)x + 0.5f, py = (float)y + 0.5f;
  float T = 1.f, acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
  bool act = inside;
  unsigned long long n_walk = 0;
  for (uint32_t base = rg.x; base < rg.y; base += (uint32_t)NB) {
    if (!__syncthreads_or(act)) break;
    const uint32_t e = base + threadIdx.x;
    if (e < rg.y) {
      const size_t rec = (size_t)j * a.M + a.list[e];
      const float4 co = reinterpret_cast<const float4*>(a.conic_opacity)[rec];
      s_co[threadIdx.x] = make_float4(-0.5f * kLog2e * co.x, -kLog2e * co.y, -0.5f * kLog2e * co.z, co.w);
      s_col[threadIdx.x] = reinterpret_cast<const float4*>(a.color_tau)[rec];
      s_mean[threadIdx.x] = reinterpret_cast<const float2*>(a.means2d)[rec];
    }
    __syncthreads();
    if (!act) continue;
    const int nbatch = (int)min((uint32_t)NB, rg.y - base);
    for (int gi = 0; gi < nbatch; ++gi) {
      if (COUNT) ++n_walk;
      const float4 co = s_co[gi];
      const float2 mu = s_mean[gi];
      const float dx = px - mu.x;
      const float dy = py - mu.y;
      const float power = quad_power(co.x, co.y, co.z, dx, dy);
      if (power > 0.f) continue;
      const float v = co.w * ex2_approx(power);
      if (!(v >= kAlphaMin)) continue;
      const float alpha = fminf(kAlphaMax, v);
      const float Tn = T * (1.f - alpha);
      if (Tn < kTMin) {
        act = false;
        break;
      }
      const float4 cl = s_col[gi];
      const float w = alpha * T;
      acc0 += cl.x * w;
      acc1 += cl.y * w;
      acc2 += cl.z * w;
      T = Tn;
    }
  }
  if (inside) {
    const int64_t o = ((int64_t)y * g.W + x) * 3;
    if (a.V[o] == j) a.out[o] = acc0 + T * a.bg[0];
    if (a.V[o + 1] == j) a.out[o + 1] = acc1 + T * a.bg[1];
    if (a.V[o + 2] == j) a.out[o + 2] = acc2 + T * a.bg[2];
  }
  if (COUNT) {
    unsigned long long c = n_walk;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) c += __shfl_down_sync(0xffffffffu, c, off);
    if ((threadIdx.x & 31) == 0 && c) {
      atomicAdd(a.eval_counter, c);
      atomicAdd(a.eval_counter + 1, c);
    }
  }
}

}  // namespace

cudaError_t launch_blend_fullframe(const PanelGeom& g, const BlendArgs& a, cudaStream_t s) {
  if ((int64_t)g.K * g.T == 0) return cudaSuccess;
  const int block = ((g.TW * g.TH + 31) / 32) * 32;
  const size_t smem = (size_t)block * (2 * sizeof(float4) + sizeof(float2));
  if (a.eval_counter)
    k_blend_fullframe<true><<<(unsigned)((int64_t)g.K * g.T), block, smem, s>>>(g, a);
  else
    k_blend_fullframe<false><<<(unsigned)((int64_t)g.K * g.T), block, smem, s>>>(g, a);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace lfd
