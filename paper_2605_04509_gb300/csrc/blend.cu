// Subpixel alpha blending with view-coherent remapping (Sec. 4.3, Eq. 9-10;
// Alg. 2 Alpha-Blend; 3DGS rules: alpha = min(0.99, o exp(-q/2)), skip
// alpha < 1/255, stop before a Gaussian that would take T below 1e-4).
//
// Work unit: one (tile t, cluster k) run of the remap table Psi. Because Psi
// sorts each tile's subpixels by view, the subpixels of cluster k form one
// contiguous run and all of them walk the same list [S_tk, E_tk). One warp
// owns one run, with no block-wide synchronisation: warps run independently.
// The warp stages the list 32 entries at a time in its own shared memory
// (conic pre-scaled by log2(e), skip threshold, opacity, colour, and the 2D
// means of every slot view of the cluster), one entry per lane.
//
// Culling per view and sub-tile. Each staged entry gets one bit per (slot
// view, sub-tile) telling whether that view's region (bounding box of
// q <= tau, one pixel of margin) meets the sub-tile; the sub-tiles are the
// tile's left and right halves (clusters of up to 16 views) or the whole
// tile (quadrants are supported as well). A 32 x 32 bit transpose across the warp
// turns the 32 entries' masks into one 32-bit list per (view, sub-tile). A
// subpixel walks only the list of its own view and sub-tile: the union over
// the cluster's views (Alg. 2) keeps the other entries in L, but they cannot
// reach alpha >= 1/255 at this subpixel, so skipping them leaves every result
// bit-identical.
//
// Subpixels. The run's subpixels are sorted by (view, sub-tile) once (a
// counting sort in the warp's shared memory); their transmittance and colour
// live in shared memory between batches. For each batch the warp takes the
// subpixels still live 32 at a time, one per lane, so lanes next to each
// other walk the same or neighbouring lists; subpixels that saturate are
// written out at once and dropped from the live list (order kept), so later
// batches keep every lane busy. An entry whose exponent lies below
// log2(1 / (255 o)) (less a 1e-4 margin) is skipped before the exp2. Entries
// are taken two at a time (the loads, quadratic forms and exponentials of the
// pair are independent) and the transmittance is then updated in list order.
// Runs are numbered cluster-major so that one cluster's attributes stay
// resident in L2 while its tiles are blended.
#include "lfd_internal.h"

namespace lfd {
namespace {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;

// Hardware approximations (hand-written PTX instructions) for the staging's
// culling bounds and skip threshold. Both only decide which list entries are
// evaluated, never a result: the skip threshold keeps a 1e-4 margin (in log2
// units) far above the approximation's error, and the box half-widths are
// widened by a relative 1e-5, so no entry that can reach alpha >= 1/255 is
// dropped and the images are the same bit for bit.
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// list entries staged per batch: one per lane (more per lane cost more shared
// memory per warp, and fewer resident warps, than they save)
constexpr int kNE = 1;
static_assert(kNE == 1, "the list entry of the next batch is fetched one per lane");
constexpr int kNB = 32 * kNE;
typedef uint32_t ListBits;  // one list of a batch: bit e = entry e
__device__ __forceinline__ int bits_first(ListBits b) { return __ffs(b) - 1; }

// sub-tiles per tile for a cluster of C views: (view, sub-tile) bits fit 32
__host__ __device__ inline int blend_subtiles(int C) { return C <= 16 ? 2 : 1; }

// Shared memory of one warp (byte offsets) for clusters of C views and runs
// of at most S subpixels (S a multiple of 8).
struct WarpSmem {
  size_t co, oc, mean, mask, info, T, acc, live, total;
};
__host__ __device__ inline WarpSmem warp_layout(int C, int S) {
  WarpSmem w;
  size_t o = 0;
  w.co = o;   o += (size_t)kNB * 16;      // float4 [kNB]: scaled conic, skip threshold
  w.oc = o;   o += (size_t)3 * kNB * 8;   // float2 [3][kNB]: (opacity, colour u)
  w.mean = o; o += (size_t)((C + 1) / 2) * kNB * 16;  // float4 [C/2][kNB]: means of views 2p, 2p + 1
  w.mask = o; o += (size_t)kNB * 4;       // u32 [kNB]: entry bits (set-up: key histogram)
  w.info = o; o += (size_t)S * 4;         // u32 [S]: packed subpixel (see pack_info)
  w.T = o;    o += (size_t)S * 4;         // float [S]: transmittance
  w.acc = o;  o += (size_t)S * 4;         // float [S]: colour so far
  w.live = o; o += ((size_t)S * 2 + 15) & ~(size_t)15;  // u16 [S]: live subpixels, in order
  w.total = (o + 15) & ~(size_t)15;
  return w;
}

// 32 x 32 bit-matrix transpose across a warp: lane i holds row i on entry and
// column i on return (bit k of the result = bit i of lane k's row).
__device__ __forceinline__ uint32_t warp_bit_transpose(uint32_t x, int lane) {
  uint32_t m = 0x0000ffffu;
#pragma unroll
  for (int j = 16; j > 0; j >>= 1, m ^= m << j) {
    const uint32_t y = __shfl_xor_sync(0xffffffffu, x, j);
    x = (lane & j) ? ((x & ~m) | ((y >> j) & m)) : ((x & m) | ((y << j) & ~m));
  }
  return x;
}

// A subpixel of a run: its position r in the run (12 bits: a run holds at
// most the 3072 subpixels of a 1024-pixel tile), channel u (2), local column
// (6) and row (6) in the tile, slot view in the cluster (5).
__device__ __forceinline__ uint32_t pack_info(int r, int u, int xl, int yl, int slot) {
  return (uint32_t)r | ((uint32_t)u << 12) | ((uint32_t)xl << 14) | ((uint32_t)yl << 20) |
         ((uint32_t)slot << 26);
}

// Blend of one (tile t, cluster k) run whose list is [rg.x, rg.y) by one
// warp, in the warp's shared memory ws (capacity S subpixels).
template <int Q, bool COUNT>
__device__ __forceinline__ void warp_blend_run(const PanelGeom& g, const BlendArgs& a, int k, int t,
                                               uint2 rg, unsigned char* ws, int S) {
  const int lane = threadIdx.x & 31;
  const unsigned full = 0xffffffffu, lt = (1u << lane) - 1u;
  const int C = g.C;
  const int L = C * Q;  // lists: bit l * Q + h for slot view l, sub-tile h
  const WarpSmem lay = warp_layout(C, S);
  float4* s_co = reinterpret_cast<float4*>(ws + lay.co);
  float2* s_oc = reinterpret_cast<float2*>(ws + lay.oc);
  float2* s_mean = reinterpret_cast<float2*>(ws + lay.mean);
  uint32_t* s_mask = reinterpret_cast<uint32_t*>(ws + lay.mask);
  uint32_t* s_info = reinterpret_cast<uint32_t*>(ws + lay.info);
  float* s_T = reinterpret_cast<float*>(ws + lay.T);
  float* s_acc = reinterpret_cast<float*>(ws + lay.acc);
  uint16_t* s_live = reinterpret_cast<uint16_t*>(ws + lay.live);

  const int s0 = a.seg[(size_t)t * (g.K + 1) + k];
  const int n = a.seg[(size_t)t * (g.K + 1) + k + 1] - s0;
  if (n <= 0) return;
  const int tx = t % g.TX, ty = t / g.TX;
  const int x0 = tx * g.TW, y0 = ty * g.TH;
  const int hw = g.TW >> 1, hh = g.TH >> 1;  // sub-tile split (local column / row)
  // pixel-centre boxes widened by one pixel: a Gaussian whose region
  // bounding box misses a box has alpha < 1/255 on every subpixel in it.
  // x: whole tile [bx0, bx1], left half [bx0, bxl], right half [bxr, bx1];
  // y likewise with the top and bottom halves.
  const float bx0 = (float)x0 + 0.5f - 1.f;
  const float bx1 = (float)min(x0 + g.TW, g.W) - 0.5f + 1.f;
  const float by0 = (float)y0 + 0.5f - 1.f;
  const float by1 = (float)min(y0 + g.TH, g.H) - 0.5f + 1.f;
  const float bxl = Q >= 2 ? (float)(x0 + hw) - 0.5f + 1.f : bx1;
  const float bxr = Q >= 2 ? (float)(x0 + hw) + 0.5f - 1.f : bx0;
  const float byt = Q == 4 ? (float)(y0 + hh) - 0.5f + 1.f : by1;
  const float byb = Q == 4 ? (float)(y0 + hh) + 0.5f - 1.f : by0;
  auto sub_of = [&](int xl, int yl) -> int {
    return (Q >= 2 && xl >= hw ? 1 : 0) + (Q == 4 && yl >= hh ? 2 : 0);
  };
  // sub-box centres and half-widths (before the Gaussian's own half-width)
  constexpr float kSlack = 1.f / 64.f;
  const float cxa = 0.5f * (bx0 + bxl), rxa0 = 0.5f * (bxl - bx0) + kSlack;
  const float cxb = 0.5f * (bxr + bx1), rxb0 = 0.5f * (bx1 - bxr) + kSlack;
  const float cya = 0.5f * (by0 + byt), rya0 = 0.5f * (byt - by0) + kSlack;
  const float cyb = 0.5f * (byb + by1), ryb0 = 0.5f * (by1 - byb) + kSlack;
  const uint32_t* psi_run = a.psi + (size_t)t * g.cap + s0;
  // write out subpixel id (packed inf) with its final state
  auto finish = [&](uint32_t inf, float T, float acc, uint32_t stop_at) {
    const int r = (int)(inf & 4095u);
    const int u = (int)((inf >> 12) & 3u);
    const int x = x0 + (int)((inf >> 14) & 63u), y = y0 + (int)((inf >> 20) & 63u);
    const float bg = u == 0 ? a.bg[0] : (u == 1 ? a.bg[1] : a.bg[2]);
    a.out[((int64_t)y * g.W + x) * 3 + u] = acc + T * bg;
    if (a.keep) a.keep[(size_t)t * g.cap + s0 + r] = make_uint2(stop_at, __float_as_uint(T));
  };

  // set-up: the run's subpixels sorted by list (slot view, sub-tile) into
  // s_live (a counting sort; the order within a list does not matter)
  int* s_hist = reinterpret_cast<int*>(s_mask);
  s_hist[lane] = 0;
  __syncwarp();
  for (int r = lane; r < n; r += 32) {
    const uint32_t e = psi_run[r];
    const int loc = (int)(e & 0xffffu);
    const int xl = (loc / 3) % g.TW, yl = (loc / 3) / g.TW;
    const int slot = (int)(e >> 16) - k * C;
    s_info[r] = pack_info(r, loc % 3, xl, yl, slot);
    const int key = slot * Q + sub_of(xl, yl);
    const int rank = atomicAdd(&s_hist[key], 1);
    s_T[r] = __int_as_float((key << 16) | rank);  // key and rank until placed
  }
  __syncwarp();
  {
    const int v = s_hist[lane];
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(full, inc, o);
      if (lane >= o) inc += y;
    }
    s_hist[lane] = inc - v;
  }
  __syncwarp();
  for (int r = lane; r < n; r += 32) {
    const int kr = __float_as_int(s_T[r]);
    s_live[s_hist[kr >> 16] + (kr & 0xffff)] = (uint16_t)r;
    s_T[r] = 1.f;
    s_acc[r] = 0.f;
  }
  __syncwarp();

  int n_live = n;
  unsigned long long n_visit = 0, n_eval = 0;
  // this lane's list entry of the next batch, fetched one batch ahead
  uint32_t gid_next = rg.x + (uint32_t)lane < rg.y ? a.list[rg.x + lane] : 0u;
  for (uint32_t base = rg.x; base < rg.y && n_live > 0; base += kNB) {
    // stage entries base + j * 32 + lane: attributes, per-view means,
    // (view, sub-tile) bits; then lane b holds list b of the batch
    ListBits col = 0;
    const uint32_t gid_here = gid_next;
    if (base + kNB + (uint32_t)lane < rg.y) gid_next = a.list[base + kNB + lane];
#pragma unroll
    for (int j = 0; j < kNE; ++j) {
      const int slot_e = j * 32 + lane;
      const uint32_t e = base + (uint32_t)slot_e;
      uint32_t mask = 0;
      if (e < rg.y) {
        const uint32_t gid = gid_here;
        const size_t rec = (size_t)k * a.M + gid;
        const float4 co = reinterpret_cast<const float4*>(a.conic_opacity)[rec];
        const float4 ct = reinterpret_cast<const float4*>(a.color_tau)[rec];
        // w: log2 of the opacity ratio at which alpha reaches 1/255 (skip below)
        s_co[slot_e] = make_float4(-0.5f * kLog2e * co.x, -kLog2e * co.y, -0.5f * kLog2e * co.z,
                                   -lg2_approx(255.f * co.w) - 1e-4f);
        s_oc[slot_e] = make_float2(co.w, ct.x);
        s_oc[kNB + slot_e] = make_float2(co.w, ct.y);
        s_oc[2 * kNB + slot_e] = make_float2(co.w, ct.z);
        const float det = co.x * co.z - co.y * co.y;
        const float rdet = __fdividef(1.f, det);
        const float hx = sqrt_approx(fmaxf(ct.w * co.z * rdet, 0.f)) * 1.00001f;
        const float hy = sqrt_approx(fmaxf(ct.w * co.x * rdet, 0.f)) * 1.00001f;
        // a view's box [mx -+ hx] x [my -+ hy] meets a sub-box iff its mean
        // lies within these thresholds (hx, hy are shared by the cluster's
        // views): x in [ax0, ax1] left half, [ax2, ax3] right half; y alike
        // as centre and half-width tests |m - c| <= r (r widened by 1/64 px,
        // above the rounding of c and of m - c on any panel of < 2^16 px)
        const float rxa = rxa0 + hx, rxb = rxb0 + hx, rya = rya0 + hy, ryb = ryb0 + hy;
        const float2* mp = reinterpret_cast<const float2*>(a.means2d) + rec * C;
        auto view_bits = [&](int l, float2 mu, bool store) {
          if (store) s_mean[((l >> 1) * kNB + slot_e) * 2 + (l & 1)] = mu;
          const bool xa = fabsf(mu.x - cxa) <= rxa;
          const bool xb = fabsf(mu.x - cxb) <= rxb;
          const bool ya = fabsf(mu.y - cya) <= rya;
          const bool yb = fabsf(mu.y - cyb) <= ryb;
          uint32_t bits;
          if (Q == 1)
            bits = (uint32_t)(xa && ya);
          else if (Q == 2)
            bits = (uint32_t)(xa && ya) | ((uint32_t)(xb && ya) << 1);
          else
            bits = (uint32_t)(xa && ya) | ((uint32_t)(xb && ya) << 1) | ((uint32_t)(xa && yb) << 2) |
                   ((uint32_t)(xb && yb) << 3);
          mask |= bits << (l * Q);
        };
        if ((C & 1) == 0) {
          // two views' means per 16-byte load
          const float4* mp4 = reinterpret_cast<const float4*>(mp);
          for (int l = 0; l < C; l += 2) {
            const float4 m4 = mp4[l >> 1];
            reinterpret_cast<float4*>(s_mean)[(l >> 1) * kNB + slot_e] = m4;
            view_bits(l, make_float2(m4.x, m4.y), false);
            view_bits(l + 1, make_float2(m4.z, m4.w), false);
          }
        } else {
          for (int l = 0; l < C; ++l) view_bits(l, mp[l], true);
        }
      }
      if (COUNT) s_mask[slot_e] = mask;
      const uint32_t cj = warp_bit_transpose(mask, lane);
      col |= (ListBits)(lane < L ? cj : 0u) << (32 * j);
    }
    __syncwarp();
    const int nbatch = (int)min((uint32_t)kNB, rg.y - base);
    int w = 0;  // live subpixels kept so far (the live list is compacted in place)
    for (int p0 = 0; p0 < n_live; p0 += 32) {
      const bool has = p0 + lane < n_live;
      const int id = has ? (int)s_live[p0 + lane] : 0;
      const uint32_t inf = s_info[id];
      float T = s_T[id], acc = s_acc[id];
      const int u = (int)((inf >> 12) & 3u);
      const int xl = (int)((inf >> 14) & 63u), yl = (int)((inf >> 20) & 63u);
      const int slot = (int)(inf >> 26);
      const float px = (float)(x0 + xl) + 0.5f, py = (float)(y0 + yl) + 0.5f;
      ListBits bits = __shfl_sync(full, col, slot * Q + sub_of(xl, yl));
      if (!has) bits = 0;
      const float2* mrow = s_mean + (slot >> 1) * kNB * 2 + (slot & 1);  // entry g at mrow[2 g]
      const float2* orow = s_oc + u * kNB;
      int stop = -1;
      while (bits) {
        const int g0 = bits_first(bits);
        bits &= bits - 1;
        const bool two = bits != 0;
        const int g1 = two ? bits_first(bits) : g0;
        bits &= bits - 1;
        const float4 c0 = s_co[g0];
        const float4 c1 = s_co[g1];
        const float2 u0 = mrow[2 * g0];
        const float2 u1 = mrow[2 * g1];
        const float p0v = quad_power(c0.x, c0.y, c0.z, px - u0.x, py - u0.y);
        const float p1v = quad_power(c1.x, c1.y, c1.z, px - u1.x, py - u1.y);
        const bool h0 = p0v <= 0.f && p0v >= c0.w;
        const bool h1 = two && p1v <= 0.f && p1v >= c1.w;
        if (!(h0 || h1)) continue;
        const float2 o0 = orow[g0];
        const float2 o1 = orow[g1];
        const float v0 = h0 ? o0.x * ex2_approx(p0v) : 0.f;
        const float v1 = h1 ? o1.x * ex2_approx(p1v) : 0.f;
        // both entries in list order without a branch per entry: entry 1
        // sees the transmittance after entry 0; the stop (rare) branches
        const bool k0 = v0 >= kAlphaMin, k1 = v1 >= kAlphaMin;
        const float a0 = fminf(kAlphaMax, v0), a1 = fminf(kAlphaMax, v1);
        const float T0 = T * (1.f - a0);
        const float Tb = k0 ? T0 : T;
        const float T1 = Tb * (1.f - a1);
        const bool s0 = k0 && T0 < kTMin;
        const bool s1 = !s0 && k1 && T1 < kTMin;
        if (k0 && !s0) acc += o0.y * a0 * T;
        if (s0 || s1) {
          stop = s0 ? g0 : g1;
          if (s1) T = Tb;
          break;
        }
        if (k1) acc += o1.y * a1 * Tb;
        T = k1 ? T1 : Tb;
      }
      const bool alive = has && stop < 0;
      if (has && stop >= 0) {
        finish(inf, T, acc, base + (uint32_t)stop);  // saturated: written now, dropped
      } else if (alive) {
        s_T[id] = T;
        s_acc[id] = acc;
      }
      if (COUNT && has) {
        // list entries walked in this batch (skipped ones included), and of
        // them the ones whose view-level bit is set (the work unit of the
        // roofline: the view's own list walked until the subpixel saturates)
        const int lim = stop >= 0 ? stop + 1 : nbatch;
        n_visit += (unsigned long long)lim;
        const uint32_t vm = ((1u << Q) - 1u) << (slot * Q);
        for (int e2 = 0; e2 < lim; ++e2) n_eval += (s_mask[e2] & vm) != 0u;
      }
      const unsigned bal = __ballot_sync(full, alive);
      if (alive) s_live[w + __popc(bal & lt)] = (uint16_t)id;
      w += __popc(bal);
    }
    n_live = w;
    __syncwarp();
  }
  // subpixels that reached the end of the list
  for (int p = lane; p < n_live; p += 32) {
    const int id = s_live[p];
    finish(s_info[id], s_T[id], s_acc[id], rg.y);
  }
  if (COUNT) {
    unsigned long long cv = n_visit, ce = n_eval;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      cv += __shfl_down_sync(full, cv, o);
      ce += __shfl_down_sync(full, ce, o);
    }
    if (lane == 0) {
      if (cv) atomicAdd(a.eval_counter, cv);
      if (ce) atomicAdd(a.eval_counter + 1, ce);
    }
  }
  __syncwarp();  // the warp's shared memory is reused by its next run
}

// One warp per (cluster, tile) run, one warp per block: a block's resources
// are released as soon as its run is done (blocks of several independent
// warps wait for the slowest one, and hold fewer warps resident).
template <int Q, bool COUNT>
__global__ void __launch_bounds__(32) k_blend(PanelGeom g, BlendArgs a, int S) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (a.P_dev && *a.P_dev > a.P_cap) return;  // capacity overflow: leave the image
  // cluster-major: one cluster's attributes stay resident in L2 while its
  // tiles are blended (tile-major order, a tile's K runs side by side, merges
  // the runs' partial image sectors in L2 but reads half as much again from
  // DRAM and was 9 % slower)
  const int nt = a.t_end - a.t_begin;
  const int k = (int)(blockIdx.x / (unsigned)nt);
  const int t = a.t_begin + (int)(blockIdx.x - (unsigned)k * (unsigned)nt);
  warp_blend_run<Q, COUNT>(g, a, k, t, a.ranges[(size_t)t * g.K + k], smem, S);
}

// Batched form: every warp of a grid sized to the GPU pulls (scene, cluster,
// tile) runs from a work counter, one run at a time, until all scenes' runs
// are done. Warp shared memory is sized for the largest cluster and run.
template <int Q>
__global__ void __launch_bounds__(256) k_blend_batch(BatchBlendArgs b, int S, int wpb, int C_max) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (b.P_dev && *b.P_dev > b.P_cap) return;  // capacity overflow: leave the images
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* ws = smem + (size_t)warp * warp_layout(C_max, S).total;
  for (;;) {
    uint32_t r = 0;
    if (lane == 0) r = atomicAdd(b.work, 1u);
    r = __shfl_sync(0xffffffffu, r, 0);
    if (r >= b.total_runs) break;
    int si = 0;
    while (si + 1 < b.n_scenes && r >= b.sc[si + 1].run_base) ++si;
    const SceneBlend& sc = b.sc[si];
    const uint32_t local = r - sc.run_base;
    const int k = (int)(local / (uint32_t)sc.g.T);
    const int t = (int)(local - (uint32_t)k * (uint32_t)sc.g.T);
    const uint2 rg = b.ranges[((size_t)si * b.T_max + t) * b.K_glob + k];
    warp_blend_run<Q, false>(sc.g, sc.a, k, t, rg, ws, S);
  }
}

// subpixel capacity of a warp for runs of up to max_segment subpixels
inline int warp_capacity(int max_segment) { return ((max(max_segment, 1) + 7) / 8) * 8; }
// warps per block of the persistent batched blend (its warps pull runs until
// none are left, so they finish together)
inline int warps_per_block(size_t per_warp) {
  return per_warp <= 12 * 1024 ? 4 : (per_warp <= 24 * 1024 ? 2 : 1);
}

template <int Q, bool COUNT>
cudaError_t launch_q(const PanelGeom& g, const BlendArgs& a, cudaStream_t s) {
  const int S = warp_capacity(a.max_segment);
  const size_t smem = warp_layout(g.C, S).total;  // one warp per block
  if (smem > 48 * 1024) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_blend<Q, COUNT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int64_t runs = (int64_t)g.K * (a.t_end - a.t_begin);
  k_blend<Q, COUNT><<<(unsigned)runs, 32, smem, s>>>(g, a, S);
  note_launches(1);
  return cudaGetLastError();
}

template <int Q>
cudaError_t launch_batch_q(const BatchBlendArgs& b, int max_segment, int C_max, cudaStream_t s) {
  const int S = warp_capacity(max_segment);
  const size_t per = warp_layout(C_max, S).total;
  const int wpb = warps_per_block(per);
  const size_t smem = per * (size_t)wpb;
  cudaError_t e =
      cudaFuncSetAttribute(k_blend_batch<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_blend_batch<Q>, 32 * wpb, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t blocks_needed = ((int64_t)b.total_runs + wpb - 1) / wpb;
  const int64_t want = (int64_t)(per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  const unsigned grid = (unsigned)(want < blocks_needed ? want : blocks_needed);
  if (grid == 0) return cudaSuccess;
  k_blend_batch<Q><<<grid, 32 * wpb, smem, s>>>(b, S, wpb, C_max);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_blend_batch(const BatchBlendArgs& b, int max_segment, int C_max,
                               int subpixels_per_thread, cudaStream_t s) {
  (void)subpixels_per_thread;  // the warp-per-run blend has no staging-depth choice
  if (b.total_runs == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(b.work, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  return blend_subtiles(C_max) == 2 ? launch_batch_q<2>(b, max_segment, C_max, s)
                                    : launch_batch_q<1>(b, max_segment, C_max, s);
}

cudaError_t launch_blend(const PanelGeom& g, const BlendArgs& args, cudaStream_t s) {
  BlendArgs a = args;
  if (a.t_end < 0 || a.t_end > g.T) a.t_end = g.T;
  if (a.t_begin < 0) a.t_begin = 0;
  if (g.K == 0 || a.t_end <= a.t_begin) return cudaSuccess;
  const int need = a.max_segment > 0 ? a.max_segment : 1;
  if (need > kMaxTileSubpixels) return cudaErrorInvalidValue;
  const int Q = blend_subtiles(g.C);
  if (a.eval_counter) return Q == 2 ? launch_q<2, true>(g, a, s) : launch_q<1, true>(g, a, s);
  return Q == 2 ? launch_q<2, false>(g, a, s) : launch_q<1, false>(g, a, s);
}

}  // namespace lfd
