// Subpixel alpha blending with view-coherent remapping (Sec. 4.3, Eq. 9-10;
// Alg. 2 Alpha-Blend; 3DGS rules: alpha = min(0.99, o exp(-q/2)), skip
// alpha < 1/255, stop before a Gaussian that would take T below 1e-4).
//
// Work unit: one (tile t, cluster k) run of the remap table Psi. Because Psi
// sorts each tile's subpixels by view, the subpixels of cluster k form one
// contiguous run and all of them walk the same list [S_tk, E_tk). One CTA
// owns one run: the list is staged in shared memory in batches of blockDim
// Gaussians (conic pre-scaled by log2(e), opacity, colour, and the 2D means
// of every slot view of the cluster), and each thread blends its subpixels
// against the staged batch; a block-wide vote ends the walk once every
// subpixel has saturated. While staging, each Gaussian gets a bit per slot
// view telling whether that view's region (bounding box of q <= tau, one
// pixel of margin) meets the tile, and per view the staged entries with that
// bit set are compacted (warp ballots) into an index list; each subpixel walks
// only its own view's list. The union over the cluster's views (Alg. 2) keeps
// the other entries in the list, but they cannot reach alpha >= 1/255 for
// this view, so skipping them leaves every result bit-identical. Means are
// staged view-major ([view][entry]) so that staging stores and per-view reads
// do not collide in shared-memory banks. An entry whose exponent lies below
// log2(1 / (255 o)) (less a 1e-4 margin) is skipped before the exp2: it cannot
// reach alpha >= 1/255. Each thread owns two subpixels of the run. Grid order
// is cluster-major so that one cluster's attributes stay resident in L2 while
// its tiles are blended.
#include "lfd_internal.h"

namespace lfd {
namespace {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int R, bool COUNT>
__global__ void __launch_bounds__(256) k_blend(PanelGeom g, BlendArgs a) {
  extern __shared__ float4 smem[];
  const int NB = blockDim.x;  // a multiple of 32
  const int NW = NB >> 5;
  const int C = g.C;
  float4* s_co = smem;        // conic * (-log2(e) / 2, -log2(e), -log2(e) / 2), opacity
  float4* s_col = smem + NB;  // colour
  float2* s_mean = reinterpret_cast<float2*>(smem + 2 * NB);        // [C][NB]
  uint16_t* s_idx = reinterpret_cast<uint16_t*>(s_mean + NB * C);   // [C][NB]
  int* s_cnt = reinterpret_cast<int*>(s_idx + ((C * NB + 1) & ~1));  // [C][NW + 1]

  const int k = blockIdx.x / g.T;
  const int t = blockIdx.x - k * g.T;
  const int s0 = a.seg[(size_t)t * (g.K + 1) + k];
  const int n = a.seg[(size_t)t * (g.K + 1) + k + 1] - s0;
  if (n <= 0) return;
  const uint2 rg = a.ranges[(size_t)t * g.K + k];
  const int tx = t % g.TX, ty = t / g.TX;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  // pixel-centre box of the tile, widened by one pixel: a Gaussian whose
  // region bounding box misses it has alpha < 1/255 on every subpixel here
  const float bx0 = (float)(tx * g.TW) + 0.5f - 1.f;
  const float bx1 = (float)min(tx * g.TW + g.TW, g.W) - 0.5f + 1.f;
  const float by0 = (float)(ty * g.TH) + 0.5f - 1.f;
  const float by1 = (float)min(ty * g.TH + g.TH, g.H) - 0.5f + 1.f;

  float px[R], py[R], T[R], acc[R];
  int slot[R], ch[R];
  int64_t oidx[R];
  bool act[R];
  unsigned long long n_visit = 0, n_eval = 0;
#pragma unroll
  for (int m = 0; m < R; ++m) {
    const int r = threadIdx.x + m * NB;
    act[m] = r < n;
    T[m] = 1.f;
    acc[m] = 0.f;
    px[m] = py[m] = 0.f;
    slot[m] = 0;
    ch[m] = 0;
    oidx[m] = 0;
    if (act[m]) {
      const uint32_t e = a.psi[(size_t)t * g.cap + s0 + r];
      const int view = (int)(e >> 16);
      const int loc = (int)(e & 0xffffu);
      const int u = loc % 3;
      const int xl = (loc / 3) % g.TW;
      const int yl = (loc / 3) / g.TW;
      const int x = tx * g.TW + xl, y = ty * g.TH + yl;
      px[m] = (float)x + 0.5f;
      py[m] = (float)y + 0.5f;
      slot[m] = view - k * C;
      ch[m] = u;
      oidx[m] = ((int64_t)y * g.W + x) * 3 + u;
    }
  }
  bool live[R];
#pragma unroll
  for (int m = 0; m < R; ++m) live[m] = act[m];

  for (uint32_t base = rg.x; base < rg.y; base += (uint32_t)NB) {
    bool any = false;
#pragma unroll
    for (int m = 0; m < R; ++m) any |= act[m];
    if (!__syncthreads_or(any)) break;
    // stage one batch: attributes, per-view means and the footprint bits
    const uint32_t e = base + threadIdx.x;
    uint32_t mask = 0;
    if (e < rg.y) {
      const uint32_t gid = a.list[e];
      const size_t rec = (size_t)k * a.M + gid;
      const float4 co = reinterpret_cast<const float4*>(a.conic_opacity)[rec];
      const float4 ct = reinterpret_cast<const float4*>(a.color_tau)[rec];
      s_co[threadIdx.x] = make_float4(-0.5f * kLog2e * co.x, -kLog2e * co.y, -0.5f * kLog2e * co.z, co.w);
      // w: log2 of the opacity ratio at which alpha reaches 1/255 (skip below)
      s_col[threadIdx.x] = make_float4(ct.x, ct.y, ct.z, -log2f(255.f * co.w) - 1e-4f);
      const float det = co.x * co.z - co.y * co.y;
      const float hx = sqrtf(fmaxf(ct.w * co.z / det, 0.f));
      const float hy = sqrtf(fmaxf(ct.w * co.x / det, 0.f));
      const float2* mp = reinterpret_cast<const float2*>(a.means2d) + rec * C;
      for (int l = 0; l < C; ++l) {
        const float2 mu = mp[l];
        s_mean[l * NB + threadIdx.x] = mu;
        const bool hit = (mu.x + hx >= bx0) && (mu.x - hx <= bx1) && (mu.y + hy >= by0) &&
                         (mu.y - hy <= by1);
        mask |= (uint32_t)hit << l;
      }
    }
    // per-view compaction: s_idx[l][..] lists, in list order, the staged
    // entries whose view-l region meets the tile
    for (int l = 0; l < C; ++l) {
      const unsigned b = __ballot_sync(0xffffffffu, (mask >> l) & 1u);
      if (lane == 0) s_cnt[l * (NW + 1) + warp] = __popc(b);
    }
    __syncthreads();
    if (threadIdx.x < C) {
      int run = 0;
      for (int w = 0; w < NW; ++w) {
        const int c = s_cnt[threadIdx.x * (NW + 1) + w];
        s_cnt[threadIdx.x * (NW + 1) + w] = run;
        run += c;
      }
      s_cnt[threadIdx.x * (NW + 1) + NW] = run;
    }
    __syncthreads();
    for (int l = 0; l < C; ++l) {
      const unsigned b = __ballot_sync(0xffffffffu, (mask >> l) & 1u);
      if ((mask >> l) & 1u) s_idx[l * NB + s_cnt[l * (NW + 1) + warp] + __popc(b & lt)] = (uint16_t)threadIdx.x;
    }
    __syncthreads();
    const int nbatch = (int)min((uint32_t)NB, rg.y - base);
#pragma unroll
    for (int m = 0; m < R; ++m) {
      if (!act[m]) continue;
      const uint16_t* idx = s_idx + slot[m] * NB;
      const int cnt = s_cnt[slot[m] * (NW + 1) + NW];
      int stop = -1;
      for (int q = 0; q < cnt; ++q) {
        const int gi = idx[q];
        if (COUNT) ++n_eval;
        const float4 co = s_co[gi];
        const float4 cl = s_col[gi];
        const float2 mu = s_mean[slot[m] * NB + gi];
        const float dx = px[m] - mu.x;
        const float dy = py[m] - mu.y;
        const float power = co.x * dx * dx + co.z * dy * dy + co.y * dx * dy;
        if (power > 0.f || power < cl.w) continue;
        const float v = co.w * ex2_approx(power);
        if (!(v >= kAlphaMin)) continue;
        const float alpha = fminf(kAlphaMax, v);
        const float Tn = T[m] * (1.f - alpha);
        if (Tn < kTMin) {
          act[m] = false;
          stop = gi;
          break;
        }
        const float c = ch[m] == 0 ? cl.x : (ch[m] == 1 ? cl.y : cl.z);
        acc[m] += c * alpha * T[m];
        T[m] = Tn;
      }
      // list entries walked in this batch, skipped ones included
      if (COUNT) n_visit += stop >= 0 ? (unsigned long long)(stop + 1) : (unsigned long long)nbatch;
    }
  }
#pragma unroll
  for (int m = 0; m < R; ++m) {
    if (!live[m]) continue;
    const float bg = ch[m] == 0 ? a.bg[0] : (ch[m] == 1 ? a.bg[1] : a.bg[2]);
    a.out[oidx[m]] = acc[m] + T[m] * bg;
  }
  if (COUNT) {
    unsigned long long cv = n_visit, ce = n_eval;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      cv += __shfl_down_sync(0xffffffffu, cv, o);
      ce += __shfl_down_sync(0xffffffffu, ce, o);
    }
    if (lane == 0) {
      if (cv) atomicAdd(a.eval_counter, cv);
      if (ce) atomicAdd(a.eval_counter + 1, ce);
    }
  }
}

template <int R>
cudaError_t launch_r(const PanelGeom& g, const BlendArgs& a, int block, cudaStream_t s) {
  const int nw = block / 32;
  const size_t smem = (size_t)block * (2 * sizeof(float4) + g.C * sizeof(float2)) +
                      (((size_t)g.C * block + 1) & ~(size_t)1) * sizeof(uint16_t) +
                      (size_t)g.C * (nw + 1) * sizeof(int);
  const unsigned grid = (unsigned)((int64_t)g.K * g.T);
  if (a.eval_counter) {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(k_blend<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_blend<R, true><<<grid, block, smem, s>>>(g, a);
    note_launches(1);
  } else {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(k_blend<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_blend<R, false><<<grid, block, smem, s>>>(g, a);
    note_launches(1);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_blend(const PanelGeom& g, const BlendArgs& a, cudaStream_t s) {
  if ((int64_t)g.K * g.T == 0) return cudaSuccess;
  const int need = a.max_segment > 0 ? a.max_segment : 1;
  int R = 2;
  while (R < 8 && (need + R - 1) / R > 256) R *= 2;
  int block = (need + R - 1) / R;
  block = ((block + 31) / 32) * 32;
  if (block > 256) return cudaErrorInvalidValue;
  switch (R) {
    case 1:
      return launch_r<1>(g, a, block, s);
    case 2:
      return launch_r<2>(g, a, block, s);
    case 4:
      return launch_r<4>(g, a, block, s);
    default:
      return launch_r<8>(g, a, block, s);
  }
}

}  // namespace lfd
