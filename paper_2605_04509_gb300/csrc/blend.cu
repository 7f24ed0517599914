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
// reach alpha >= 1/255. A thread owns R subpixels of the run (R = 2 unless
// the plan sets another staging depth) and takes its view's entries two at a
// time: the loads, quadratic forms and exponentials of the pair are
// independent, and the transmittance is then updated in list order. Grid
// order is cluster-major so that one cluster's attributes stay resident in L2
// while its tiles are blended.
#include "lfd_internal.h"

namespace lfd {
namespace {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;

// Blend of one (tile t, cluster k) run whose list is [rg.x, rg.y). Called by
// every thread of the block (it synchronises the block); returns uniformly.
template <int R, bool COUNT>
__device__ __forceinline__ void blend_run(const PanelGeom& g, const BlendArgs& a, int k, int t,
                                          uint2 rg, float4* smem) {
  const int NB = blockDim.x;  // a multiple of 32
  const int NW = NB >> 5;
  const int C = g.C;
  float4* s_co = smem;  // conic * (-log2(e) / 2, -log2(e), -log2(e) / 2), skip threshold
  float2* s_oc = reinterpret_cast<float2*>(smem + NB);              // [3][NB] (opacity, colour u)
  float2* s_mean = reinterpret_cast<float2*>(smem + 2 * NB) + NB;   // [C][NB]
  uint16_t* s_idx = reinterpret_cast<uint16_t*>(s_mean + NB * C);   // [C][NB]
  int* s_cnt = reinterpret_cast<int*>(s_idx + ((C * NB + 1) & ~1));  // [C][NW + 1]

  const int s0 = a.seg[(size_t)t * (g.K + 1) + k];
  const int n = a.seg[(size_t)t * (g.K + 1) + k + 1] - s0;
  if (n <= 0) return;
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
  uint32_t stop_at[R];  // list index where the walk stopped
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
    stop_at[m] = rg.y;
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
      // w: log2 of the opacity ratio at which alpha reaches 1/255 (skip below)
      s_co[threadIdx.x] = make_float4(-0.5f * kLog2e * co.x, -kLog2e * co.y, -0.5f * kLog2e * co.z,
                                      -log2f(255.f * co.w) - 1e-4f);
      s_oc[threadIdx.x] = make_float2(co.w, ct.x);
      s_oc[NB + threadIdx.x] = make_float2(co.w, ct.y);
      s_oc[2 * NB + threadIdx.x] = make_float2(co.w, ct.z);
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
      int stop = -1, stop_q = -1;
      const float2* mrow = s_mean + slot[m] * NB;
      const float2* orow = s_oc + ch[m] * NB;
      // Entries are taken two at a time: their loads, quadratic forms and
      // exponentials are independent; the transmittance update stays in
      // list order, one entry after the other.
      auto apply = [&](int gi, float v, float c) -> bool {
        if (!(v >= kAlphaMin)) return false;
        const float alpha = fminf(kAlphaMax, v);
        const float Tn = T[m] * (1.f - alpha);
        if (Tn < kTMin) {
          act[m] = false;
          stop = gi;
          return true;
        }
        acc[m] += c * alpha * T[m];
        T[m] = Tn;
        return false;
      };
      int q = 0;
      for (; q + 2 <= cnt; q += 2) {
        const int g0 = idx[q], g1 = idx[q + 1];
        const float4 c0 = s_co[g0];
        const float4 c1 = s_co[g1];
        const float2 u0 = mrow[g0];
        const float2 u1 = mrow[g1];
        const float dx0 = px[m] - u0.x, dy0 = py[m] - u0.y;
        const float dx1 = px[m] - u1.x, dy1 = py[m] - u1.y;
        const float p0 = quad_power(c0.x, c0.y, c0.z, dx0, dy0);
        const float p1 = quad_power(c1.x, c1.y, c1.z, dx1, dy1);
        const bool h0 = p0 <= 0.f && p0 >= c0.w;
        const bool h1 = p1 <= 0.f && p1 >= c1.w;
        if (!(h0 || h1)) continue;
        const float2 o0 = orow[g0];
        const float2 o1 = orow[g1];
        const float v0 = h0 ? o0.x * ex2_approx(p0) : 0.f;
        const float v1 = h1 ? o1.x * ex2_approx(p1) : 0.f;
        if (apply(g0, v0, o0.y)) {
          stop_q = q;
          break;
        }
        if (apply(g1, v1, o1.y)) {
          stop_q = q + 1;
          break;
        }
      }
      if (stop < 0 && q < cnt) {
        const int gi = idx[q];
        const float4 co = s_co[gi];
        const float2 mu = mrow[gi];
        const float dx = px[m] - mu.x;
        const float dy = py[m] - mu.y;
        const float power = quad_power(co.x, co.y, co.z, dx, dy);
        if (power <= 0.f && power >= co.w) {
          const float2 oc = orow[gi];
          if (apply(gi, oc.x * ex2_approx(power), oc.y)) stop_q = q;
        }
      }
      if (stop >= 0) stop_at[m] = base + (uint32_t)stop;
      if (COUNT) n_eval += stop_q >= 0 ? (unsigned long long)(stop_q + 1) : (unsigned long long)cnt;
      // list entries walked in this batch, skipped ones included
      if (COUNT) n_visit += stop >= 0 ? (unsigned long long)(stop + 1) : (unsigned long long)nbatch;
    }
  }
#pragma unroll
  for (int m = 0; m < R; ++m) {
    if (!live[m]) continue;
    const float bg = ch[m] == 0 ? a.bg[0] : (ch[m] == 1 ? a.bg[1] : a.bg[2]);
    a.out[oidx[m]] = acc[m] + T[m] * bg;
    if (a.keep)
      a.keep[(size_t)t * g.cap + s0 + threadIdx.x + m * NB] = make_uint2(stop_at[m], __float_as_uint(T[m]));
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

template <int R, bool COUNT>
__global__ void __launch_bounds__(256) k_blend(PanelGeom g, BlendArgs a) {
  extern __shared__ float4 smem[];
  if (a.P_dev && *a.P_dev > a.P_cap) return;  // capacity overflow: leave the image
  const int nt = a.t_end - a.t_begin;
  const int k = blockIdx.x / nt;
  const int t = a.t_begin + (blockIdx.x - k * nt);
  blend_run<R, COUNT>(g, a, k, t, a.ranges[(size_t)t * g.K + k], smem);
}

// Batched, persistent form: a grid sized to the GPU pulls (scene, cluster,
// tile) runs from a work counter, kBatchChunk consecutive runs at a time (one
// atomic and two barriers per chunk, not per run: most runs of a large panel
// are short), until all scenes' runs are done.
constexpr uint32_t kBatchChunk = 8;

// (R <= 2: at most 48 registers, like the single-scene blend, so that eight
// 160-thread blocks fit an SM rather than six)
template <int R>
__global__ void __launch_bounds__(256, R <= 2 ? 5 : 2) k_blend_batch(BatchBlendArgs b) {
  extern __shared__ float4 smem[];
  __shared__ uint32_t s_run;
  if (b.P_dev && *b.P_dev > b.P_cap) return;  // capacity overflow: leave the images
  for (;;) {
    if (threadIdx.x == 0) s_run = atomicAdd(b.work, kBatchChunk);
    __syncthreads();
    const uint32_t r0 = s_run;
    __syncthreads();
    if (r0 >= b.total_runs) break;
    const uint32_t r1 = min(r0 + kBatchChunk, b.total_runs);
    int si = 0;
    for (uint32_t r = r0; r < r1; ++r) {
      while (si + 1 < b.n_scenes && r >= b.sc[si + 1].run_base) ++si;
      const SceneBlend& sc = b.sc[si];
      const uint32_t local = r - sc.run_base;
      const int k = (int)(local / (uint32_t)sc.g.T);
      const int t = (int)(local - (uint32_t)k * (uint32_t)sc.g.T);
      const uint2 rg = b.ranges[((size_t)si * b.T_max + t) * b.K_glob + k];
      blend_run<R, false>(sc.g, sc.a, k, t, rg, smem);
      __syncthreads();  // the next run restages shared memory
    }
  }
}

size_t blend_smem_bytes(int C, int block) {
  const int nw = block / 32;
  return (size_t)block * (sizeof(float4) + 3 * sizeof(float2) + C * sizeof(float2)) +
         (((size_t)C * block + 1) & ~(size_t)1) * sizeof(uint16_t) + (size_t)C * (nw + 1) * sizeof(int);
}

template <int R>
cudaError_t launch_r(const PanelGeom& g, const BlendArgs& a, int block, cudaStream_t s) {
  const size_t smem = blend_smem_bytes(g.C, block);
  const unsigned grid = (unsigned)((int64_t)g.K * (a.t_end - a.t_begin));
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


template <int R>
cudaError_t launch_batch_r(const BatchBlendArgs& b, int block, int C_max, cudaStream_t s) {
  const size_t smem = blend_smem_bytes(C_max, block);
  cudaError_t e =
      cudaFuncSetAttribute(k_blend_batch<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_blend_batch<R>, block, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (int64_t)(per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  const unsigned grid = (unsigned)(want < (int64_t)b.total_runs ? want : (int64_t)b.total_runs);
  if (grid == 0) return cudaSuccess;
  k_blend_batch<R><<<grid, block, smem, s>>>(b);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace

// Subpixels per thread: the requested count when its block fits 256 threads,
// else the smallest power of two from 2 up that does.
static int choose_r(int need, int requested) {
  if (requested > 0 && (need + requested - 1) / requested <= 256) return requested;
  int R = 2;
  while (R < 8 && (need + R - 1) / R > 256) R *= 2;
  return R;
}

cudaError_t launch_blend_batch(const BatchBlendArgs& b, int max_segment, int C_max,
                               int subpixels_per_thread, cudaStream_t s) {
  if (b.total_runs == 0) return cudaSuccess;
  const int need = max_segment > 0 ? max_segment : 1;
  const int R = choose_r(need, subpixels_per_thread);
  int block = (need + R - 1) / R;
  block = ((block + 31) / 32) * 32;
  if (block > 256) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(b.work, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  switch (R) {
    case 1:
      return launch_batch_r<1>(b, block, C_max, s);
    case 2:
      return launch_batch_r<2>(b, block, C_max, s);
    case 4:
      return launch_batch_r<4>(b, block, C_max, s);
    default:
      return launch_batch_r<8>(b, block, C_max, s);
  }
}

cudaError_t launch_blend(const PanelGeom& g, const BlendArgs& args, cudaStream_t s) {
  BlendArgs a = args;
  if (a.t_end < 0 || a.t_end > g.T) a.t_end = g.T;
  if (a.t_begin < 0) a.t_begin = 0;
  if (g.K == 0 || a.t_end <= a.t_begin) return cudaSuccess;
  const int need = a.max_segment > 0 ? a.max_segment : 1;
  const int R = choose_r(need, a.subpixels_per_thread);
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
