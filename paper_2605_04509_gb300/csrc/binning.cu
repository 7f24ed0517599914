// Key generation with cross-view coherent attribute reuse (Sec. 4.2 "Key
// Generation"; Alg. 2 GenerateKeys; Eq. 11) and range identification
// (Sec. 4.2 "Sorting": the list of (tile t, cluster k) is [S_tk, E_tk)).
//
// Tile-bin rule. The region of Gaussian i in view j is the ellipse
// {p : q(p - mu_ij) <= tau_ik} with q the conic of the representative view;
// it holds exactly the pixel centres where alpha >= 1/255 (Eq. 10). For every
// tile row, the exact horizontal extent of the ellipse over the row's band of
// pixel-centre heights is taken (the extreme lies where the ellipse's right-
// or leftmost point, clamped into the band, sits); a tile is hit when a
// pixel-centre column inside that extent falls in it. The cluster's tiles are
// the union over its views (Alg. 2: tiles overlapping at least one view).
// Every floating-point step below is an IEEE float32 operation with
// round-to-nearest (the _rn intrinsics; no contraction) in a fixed order, so
// the integer outcome (which tiles) is reproducible bit for bit.
#include "lfd_internal.h"

namespace lfd {
namespace {

struct BinQ {
  float a, b, c, tau, det, hx, hy, ys, ia;
};

struct BinV {
  float mx, my, bx0, bx1;
  int y0, y1;
  bool valid;
};

__device__ __forceinline__ bool bin_prep(float a, float b, float c, float tau, BinQ& g) {
  if (!isfinite(a) || !isfinite(b) || !isfinite(c) || !isfinite(tau)) return false;
  if (!(tau >= 0.f) || !(a > 0.f) || !(c > 0.f)) return false;
  const float ac = __fmul_rn(a, c);
  const float bb = __fmul_rn(b, b);
  const float det = __fsub_rn(ac, bb);
  if (!(det > 0.f)) return false;
  g.a = a;
  g.b = b;
  g.c = c;
  g.tau = tau;
  g.det = det;
  const float ta = __fmul_rn(tau, a);
  const float tc = __fmul_rn(tau, c);
  g.hy = __fsqrt_rn(__fdiv_rn(ta, det));
  g.hx = __fsqrt_rn(__fdiv_rn(tc, det));
  const float dc = __fmul_rn(det, c);
  const float r = __fsqrt_rn(__fdiv_rn(tau, dc));
  g.ys = __fmul_rn(b, r);
  g.ia = __fdiv_rn(1.f, a);
  return true;
}

// pixel rows / columns whose centre lies inside the ellipse's bounding box
__device__ __forceinline__ void bin_view(const BinQ& g, float mx, float my, int W, int H,
                                         BinV& v) {
  v.valid = false;
  if (!isfinite(mx) || !isfinite(my)) return;
  const float ylo = __fsub_rn(my, g.hy);
  const float yhi = __fadd_rn(my, g.hy);
  float fy0 = ceilf(__fsub_rn(ylo, 0.5f));
  float fy1 = floorf(__fsub_rn(yhi, 0.5f));
  fy0 = fmaxf(fy0, 0.f);
  fy1 = fminf(fy1, (float)(H - 1));
  const float xlo = __fsub_rn(mx, g.hx);
  const float xhi = __fadd_rn(mx, g.hx);
  float fx0 = ceilf(__fsub_rn(xlo, 0.5f));
  float fx1 = floorf(__fsub_rn(xhi, 0.5f));
  fx0 = fmaxf(fx0, 0.f);
  fx1 = fminf(fx1, (float)(W - 1));
  if (!(fy0 <= fy1) || !(fx0 <= fx1)) return;
  v.valid = true;
  v.mx = mx;
  v.my = my;
  v.y0 = (int)fy0;
  v.y1 = (int)fy1;
  v.bx0 = fx0;
  v.bx1 = fx1;
}

// tile-column interval [tx0, tx1] of view v in tile row ty
__device__ __forceinline__ bool bin_row(const BinQ& g, const BinV& v, int ty, int TH, uint32_t tw_magic,
                                        int& tx0, int& tx1) {
  if (!v.valid) return false;
  const int ya = max(ty * TH, v.y0);
  const int yb = min(ty * TH + TH - 1, v.y1);
  if (ya > yb) return false;
  const float lo = __fsub_rn(__fadd_rn((float)ya, 0.5f), v.my);
  const float hi = __fsub_rn(__fadd_rn((float)yb, 0.5f), v.my);
  const float dR = fminf(fmaxf(-g.ys, lo), hi);
  const float dL = fminf(fmaxf(g.ys, lo), hi);
  const float at = __fmul_rn(g.a, g.tau);
  const float eR = __fmul_rn(g.det, dR);
  const float wR = __fsqrt_rn(fmaxf(__fsub_rn(at, __fmul_rn(eR, dR)), 0.f));
  const float eL = __fmul_rn(g.det, dL);
  const float wL = __fsqrt_rn(fmaxf(__fsub_rn(at, __fmul_rn(eL, dL)), 0.f));
  const float xR = __fadd_rn(v.mx, __fmul_rn(__fsub_rn(wR, __fmul_rn(g.b, dR)), g.ia));
  const float xL = __fadd_rn(v.mx, __fmul_rn(__fsub_rn(-wL, __fmul_rn(g.b, dL)), g.ia));
  const float fx0 = fmaxf(ceilf(__fsub_rn(xL, 0.5f)), v.bx0);
  const float fx1 = fminf(floorf(__fsub_rn(xR, 0.5f)), v.bx1);
  if (!(fx0 <= fx1)) return false;
  tx0 = (int)__umulhi((unsigned)(int)fx0, tw_magic);
  tx1 = (int)__umulhi((unsigned)(int)fx1, tw_magic);
  return true;
}

// Row and tile-column range of the cluster's union (bounding boxes).
__device__ __forceinline__ void bin_extent(const PanelGeom& pg, const BinQ& q,
                                           const float2* __restrict__ means, int& ty0, int& ty1,
                                           int& c0, int& c1) {
  ty0 = INT_MAX;
  ty1 = -1;
  c0 = INT_MAX;
  c1 = -1;
  for (int l = 0; l < pg.C; ++l) {
    const float2 m = means[l];
    BinV v;
    bin_view(q, m.x, m.y, pg.W, pg.H, v);
    if (!v.valid) continue;
    ty0 = min(ty0, (int)__umulhi((unsigned)v.y0, pg.th_magic));
    ty1 = max(ty1, (int)__umulhi((unsigned)v.y1, pg.th_magic));
    c0 = min(c0, (int)__umulhi((unsigned)(int)v.bx0, pg.tw_magic));
    c1 = max(c1, (int)__umulhi((unsigned)(int)v.bx1, pg.tw_magic));
  }
}

// The union of the cluster's tiles, row by row and 64 tile columns at a time:
// on_mask(ty, w0, mask) gets the tiles w0 + bit of row ty, rows and windows in
// ascending order. Returns the tile count.
template <typename OnMask>
__device__ __forceinline__ uint32_t bin_rows(const PanelGeom& pg, const BinQ& q,
                                             const float2* __restrict__ means, int ty0, int ty1,
                                             int c0, int c1, OnMask on_mask) {
  uint32_t n = 0;
  for (int ty = ty0; ty <= ty1; ++ty) {
    for (int w0 = c0; w0 <= c1; w0 += 64) {
      unsigned long long mask = 0ull;
      for (int l = 0; l < pg.C; ++l) {
        const float2 m = means[l];
        BinV v;
        bin_view(q, m.x, m.y, pg.W, pg.H, v);
        int a, b;
        if (!bin_row(q, v, ty, pg.TH, pg.tw_magic, a, b)) continue;
        a = max(a, w0);
        b = min(b, w0 + 63);
        if (a > b) continue;
        const int len = b - a + 1;
        const unsigned long long bits = len == 64 ? ~0ull : ((1ull << len) - 1ull);
        mask |= bits << (a - w0);
      }
      n += __popcll(mask);
      on_mask(ty, w0, mask);
    }
  }
  return n;
}

// Walk the union of the cluster's tiles in ascending tile id; calls emit(t).
template <typename Emit>
__device__ __forceinline__ uint32_t bin_union(const PanelGeom& pg, const BinQ& q,
                                              const float2* __restrict__ means, Emit emit) {
  int ty0, ty1, c0, c1;
  bin_extent(pg, q, means, ty0, ty1, c0, c1);
  return bin_rows(pg, q, means, ty0, ty1, c0, c1, [&](int ty, int w0, unsigned long long mask) {
    while (mask) {
      const int bit = __ffsll((long long)mask) - 1;
      mask &= mask - 1ull;
      emit(ty * pg.TX + w0 + bit);
    }
  });
}

// Compact record of an item's union written by the count pass so that the
// emit pass need not redo the geometry: header = ty0 | c0 << 16 | rows << 32
// | overflow << 40, then one 64-tile mask per row. Items whose union spans
// more than kDescRows rows or 64 tile columns are marked overflow and redone.
constexpr int kDescRows = 15;
struct __align__(16) BinDesc {
  unsigned long long header;
  unsigned long long mask[kDescRows];
};
static_assert(sizeof(BinDesc) == kBinDescBytes, "descriptor size");

__global__ void k_item_keys(PanelGeom g, int64_t M, const float* __restrict__ depth,
                            const float4* __restrict__ color_tau, uint64_t* __restrict__ keys,
                            uint32_t* __restrict__ vals) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= (int64_t)g.K * M) return;
  const uint64_t k = (uint64_t)((uint32_t)r / (uint32_t)M);  // K M < 2^32
  const float tau = color_tau[r].w;
  const uint32_t d = tau >= 0.f ? __float_as_uint(depth[r]) : 0xffffffffu;
  keys[r] = ((k + (uint64_t)g.cluster_base) << 32) | d;
  vals[r] = (uint32_t)r;
}

__device__ __forceinline__ BinQ shfl_q(const BinQ& q, int src) {
  BinQ o;
  o.a = __shfl_sync(0xffffffffu, q.a, src);
  o.b = __shfl_sync(0xffffffffu, q.b, src);
  o.c = __shfl_sync(0xffffffffu, q.c, src);
  o.tau = __shfl_sync(0xffffffffu, q.tau, src);
  o.det = __shfl_sync(0xffffffffu, q.det, src);
  o.hx = __shfl_sync(0xffffffffu, q.hx, src);
  o.hy = __shfl_sync(0xffffffffu, q.hy, src);
  o.ys = __shfl_sync(0xffffffffu, q.ys, src);
  o.ia = __shfl_sync(0xffffffffu, q.ia, src);
  return o;
}

// Exclusive prefix over the warp's lanes; *total receives the sum.
__device__ __forceinline__ int warp_exclusive(int v, int lane, int* total) {
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  *total = __shfl_sync(0xffffffffu, incl, 31);
  return incl - v;
}

// Lane of the warp owning work unit u, given each lane's first unit
// (non-decreasing over lanes): the last lane whose first unit is <= u.
__device__ __forceinline__ int unit_owner(int ubase, int u) {
  int j = 0;
#pragma unroll
  for (int st = 16; st > 0; st >>= 1) {
    const int cand = j + st;
    const int ub = __shfl_sync(0xffffffffu, ubase, cand & 31);
    if (cand < 32 && ub <= u) j = cand;
  }
  return j;
}

constexpr int kBinWarps = 4;

// Tile counts (and union descriptors) of the items. Each warp takes 32
// items; their tile rows are dealt out to the lanes as separate work units,
// so a large Gaussian does not hold up its warp. A unit unites the cluster's
// views over one tile row. Items whose union is wider than 64 tile columns
// are walked by their own lane. Each item's per-view boxes (bin_view) are
// computed once by its own lane and kept in shared memory for the units.
// Per-(item, view) boxes kept in shared memory field by field,
// [field][view][item of the block], so that lanes reading different items'
// boxes of one view hit consecutive words (no bank conflicts).
constexpr int kBoxFields = 6;  // mx, my, bx0, bx1, y0, y1 (y0 > y1: not seen)

// One block of the count pass: items [blk * 32 kBinWarps, ...) of one scene.
__device__ __forceinline__ void bin_count_block(const PanelGeom& g, int64_t M,
                                                const float2* __restrict__ means2d,
                                                const float4* __restrict__ conic_opacity,
                                                const float4* __restrict__ color_tau,
                                                const uint32_t* __restrict__ order,
                                                const uint32_t* __restrict__ dest, int64_t n_items,
                                                uint32_t* __restrict__ counts,
                                                BinDesc* __restrict__ desc, int64_t blk) {
  __shared__ uint32_t s_n[kBinWarps][32];
  extern __shared__ float s_box[];  // [kBoxFields][C][32 * kBinWarps]
  const int64_t s = blk * (32 * kBinWarps) + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool in = s < n_items;
  uint32_t r = 0;
  BinQ q = {};
  bool ok = false;
  int ty0 = INT_MAX, ty1 = -1, c0 = INT_MAX, c1 = -1;
  constexpr int kItems = 32 * kBinWarps;
  auto box = [&](int f, int l, int item) -> float& { return s_box[(f * g.C + l) * kItems + item]; };
  const int my_item = warp * 32 + lane;
  // where the item's count and descriptor go: its emission position
  int64_t o = s;
  if (in) {
    r = order ? order[s] : (uint32_t)s;
    if (dest) o = dest[r];
    const float4 co = conic_opacity[r];
    ok = bin_prep(co.x, co.y, co.z, color_tau[r].w, q);
  }
  if (ok) {
    // bin_extent, keeping each view's box
    const float2* mr = means2d + (size_t)r * g.C;
    for (int l = 0; l < g.C; ++l) {
      const float2 m = mr[l];
      BinV v;
      bin_view(q, m.x, m.y, g.W, g.H, v);
      box(0, l, my_item) = v.mx;
      box(1, l, my_item) = v.my;
      box(2, l, my_item) = v.bx0;
      box(3, l, my_item) = v.bx1;
      box(4, l, my_item) = __int_as_float(v.valid ? v.y0 : 1);
      box(5, l, my_item) = __int_as_float(v.valid ? v.y1 : 0);
      if (!v.valid) continue;
      ty0 = min(ty0, (int)__umulhi((unsigned)v.y0, g.th_magic));
      ty1 = max(ty1, (int)__umulhi((unsigned)v.y1, g.th_magic));
      c0 = min(c0, (int)__umulhi((unsigned)(int)v.bx0, g.tw_magic));
      c1 = max(c1, (int)__umulhi((unsigned)(int)v.bx1, g.tw_magic));
    }
  }
  const int rows = ok && ty1 >= ty0 ? ty1 - ty0 + 1 : 0;
  const bool wide = rows > 0 && c1 - c0 >= 64;
  const bool fits = rows <= kDescRows && !wide;
  s_n[warp][lane] = 0;
  uint32_t n_self = 0;
  if (wide)
    n_self = bin_rows(g, q, means2d + (size_t)r * g.C, ty0, ty1, c0, c1,
                      [](int, int, unsigned long long) {});
  int U;
  const int ubase = warp_exclusive(wide ? 0 : rows, lane, &U);
  __syncwarp();
  for (int b = 0; b < U; b += 32) {
    const int u = b + lane;
    const int j = unit_owner(ubase, u);
    const int rr = u - __shfl_sync(0xffffffffu, ubase, j);
    const BinQ qj = shfl_q(q, j);
    const int ty0j = __shfl_sync(0xffffffffu, ty0, j);
    const int c0j = __shfl_sync(0xffffffffu, c0, j);
    const bool fitsj = __shfl_sync(0xffffffffu, fits, j);
    const int64_t oj = (int64_t)__shfl_sync(0xffffffffu, (unsigned long long)o, j);
    if (u < U) {
      const int item_j = warp * 32 + j;
      const int ty = ty0j + rr;
      unsigned long long mask = 0ull;
      for (int l = 0; l < g.C; ++l) {
        BinV v;
        v.mx = box(0, l, item_j);
        v.my = box(1, l, item_j);
        v.bx0 = box(2, l, item_j);
        v.bx1 = box(3, l, item_j);
        v.y0 = __float_as_int(box(4, l, item_j));
        v.y1 = __float_as_int(box(5, l, item_j));
        v.valid = v.y0 <= v.y1;
        int a, bb;
        if (!bin_row(qj, v, ty, g.TH, g.tw_magic, a, bb)) continue;
        const int len = bb - a + 1;
        const unsigned long long bits = len == 64 ? ~0ull : ((1ull << len) - 1ull);
        mask |= bits << (a - c0j);
      }
      atomicAdd(&s_n[warp][j], (uint32_t)__popcll(mask));
      if (desc && fitsj) desc[oj].mask[rr] = mask;
    }
  }
  __syncwarp();
  if (in) {
    counts[o] = wide ? n_self : s_n[warp][lane];
    if (desc)
      desc[o].header = rows == 0 ? 0ull
                                 : ((unsigned long long)ty0 | ((unsigned long long)c0 << 16) |
                                    ((unsigned long long)rows << 32) |
                                    ((unsigned long long)(fits ? 0 : 1) << 40));
  }
}

__global__ void __launch_bounds__(32 * kBinWarps)
    k_bin_count(PanelGeom g, int64_t M, const float2* __restrict__ means2d,
                const float4* __restrict__ conic_opacity, const float4* __restrict__ color_tau,
                const uint32_t* __restrict__ order, const uint32_t* __restrict__ dest,
                int64_t n_items, uint32_t* __restrict__ counts, BinDesc* __restrict__ desc) {
  bin_count_block(g, M, means2d, conic_opacity, color_tau, order, dest, n_items, counts, desc,
                  blockIdx.x);
}

// Scene of block blk of a folded batch launch (scenes own consecutive blocks).
__device__ __forceinline__ int scene_of_block(const BatchBins& bb, uint32_t blk) {
  int s = 0;
  while (s + 1 < bb.n_scenes && blk >= bb.sc[s + 1].blk_off) ++s;
  return s;
}

// The count pass of every scene of a batch in one launch.
__global__ void __launch_bounds__(32 * kBinWarps)
    k_bin_count_batch(BatchBins bb, const uint32_t* __restrict__ dest, uint32_t* __restrict__ counts,
                      BinDesc* __restrict__ desc) {
  const SceneBins& sc = bb.sc[scene_of_block(bb, blockIdx.x)];
  bin_count_block(sc.g, sc.M, reinterpret_cast<const float2*>(sc.means2d),
                  reinterpret_cast<const float4*>(sc.conic_opacity),
                  reinterpret_cast<const float4*>(sc.color_tau), nullptr, dest + sc.off, sc.n,
                  counts + sc.off, desc + sc.off, blockIdx.x - sc.blk_off);
}

__global__ void k_bin_emit(PanelGeom g, int64_t M, const float2* __restrict__ means2d,
                           const float4* __restrict__ conic_opacity,
                           const float4* __restrict__ color_tau, const float* __restrict__ depth,
                           const uint32_t* __restrict__ order, int64_t n_items,
                           const uint32_t* __restrict__ offsets, uint32_t* __restrict__ keys32,
                           uint64_t* __restrict__ keys64, uint32_t* __restrict__ vals,
                           const BinDesc* __restrict__ desc) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_items) return;
  const uint32_t r = order ? order[s] : (uint32_t)s;
  const uint32_t k = r / (uint32_t)M;
  const uint32_t i = (uint32_t)(r - (uint64_t)k * M);
  uint32_t pos = offsets[s];
  if (desc) {
    const unsigned long long h = desc[s].header;
    if (!((h >> 40) & 1ull)) {
      const int ty0 = (int)(h & 0xffffull), c0 = (int)((h >> 16) & 0xffffull);
      const int rows = (int)((h >> 32) & 0xffull);
      const uint64_t lo = keys64 ? (((uint64_t)k << 32) | __float_as_uint(depth[r])) : 0ull;
      for (int rr = 0; rr < rows; ++rr) {
        unsigned long long mask = desc[s].mask[rr];
        while (mask) {
          const int bit = __ffsll((long long)mask) - 1;
          mask &= mask - 1ull;
          const uint32_t t = (uint32_t)((ty0 + rr) * g.TX + c0 + bit);
          if (keys64)
            keys64[pos] = ((uint64_t)t << (32 + g.bit_k)) | lo;
          else
            keys32[pos] = (t << g.bit_k) | k;
          vals[pos] = i;
          ++pos;
        }
      }
      return;
    }
  }
  const float4 co = conic_opacity[r];
  BinQ q;
  if (!bin_prep(co.x, co.y, co.z, color_tau[r].w, q)) return;
  if (keys64) {
    const uint64_t lo = ((uint64_t)k << 32) | __float_as_uint(depth[r]);
    const int shift = 32 + g.bit_k;
    bin_union(g, q, means2d + (size_t)r * g.C, [&](int t) {
      keys64[pos] = ((uint64_t)t << shift) | lo;
      vals[pos] = i;
      ++pos;
    });
  } else {
    bin_union(g, q, means2d + (size_t)r * g.C, [&](int t) {
      keys32[pos] = ((uint32_t)t << g.bit_k) | k;
      vals[pos] = i;
      ++pos;
    });
  }
}

// Emission from the count pass's union descriptors (indexed by item r). Each
// lane expands its own item's tiles (from the descriptor, or from the
// geometry when the union did not fit one) into a per-warp staging buffer in
// shared memory at the item's offset relative to the warp's first item; the
// warp then copies the buffer out with consecutive lanes on consecutive
// addresses, so the global stores coalesce. Warps whose items hold more
// pairs than the buffer write straight to global memory. Positions and
// contents equal the plain per-item emission's.
constexpr int kEmitWarps = 4;

template <typename KeyT>
struct EmitCap {
  static constexpr int value = (6144 / (int)(sizeof(KeyT) + 4)) & ~31;  // ~24 KB per block
};

// One block of the emit pass: items [blk * 32 kEmitWarps, ...) of one scene.
template <typename KeyT>
__device__ __forceinline__ void bin_emit_block(
    const PanelGeom& g, int64_t M, const float2* __restrict__ means2d,
    const float4* __restrict__ conic_opacity, const float4* __restrict__ color_tau,
    const float* __restrict__ depth, const uint32_t* __restrict__ order, int64_t n_items,
    const uint32_t* __restrict__ counts, const uint32_t* __restrict__ offsets, KeyT* __restrict__ keys,
    uint32_t* __restrict__ vals, const BinDesc* __restrict__ desc,
    const unsigned long long* __restrict__ P_dev, unsigned long long P_cap, uint32_t* __restrict__ err,
    int64_t blk) {
  constexpr int CAP = EmitCap<KeyT>::value;
  constexpr bool kWide = sizeof(KeyT) == 8;
  __shared__ KeyT s_key[kEmitWarps][CAP];
  __shared__ uint32_t s_val[kEmitWarps][CAP];
  const int64_t s = blk * (32 * kEmitWarps) + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (P_dev && *P_dev > P_cap) {  // more pairs than the buffers hold: write nothing
    if (s == 0) atomicOr(err, 2u);
    return;
  }
  const bool in = s < n_items;
  uint32_t r = 0, n = 0, pos = 0;
  unsigned long long h = 0ull;
  if (in) {
    r = order ? order[s] : (uint32_t)s;
    n = counts[s];
    pos = offsets[s];
    if (n) h = desc[s].header;
  }
  const unsigned valid = __ballot_sync(0xffffffffu, in);
  if (!valid) return;
  const int last = 31 - __clz((int)valid);
  const uint32_t wbase = __shfl_sync(0xffffffffu, pos, 0);
  const uint32_t wend = __shfl_sync(0xffffffffu, pos + n, last);
  const uint32_t total = wend - wbase;
  const bool staged = total <= (uint32_t)CAP;
  KeyT* kdst = staged ? &s_key[warp][0] : keys;
  uint32_t* vdst = staged ? &s_val[warp][0] : vals;
  const uint32_t shift_out = staged ? wbase : 0u;
  const int shift = kWide ? 32 + g.bit_k : g.bit_k;
  // unions that did not fit a descriptor: the owner lane redoes the geometry
  const bool redo = in && n && ((h >> 40) & 1ull);
  if (redo) {
    const uint32_t k = r / (uint32_t)M;  // K M < 2^32
    const uint32_t i = (uint32_t)(r - (uint64_t)k * M);
    const uint64_t lo = kWide ? (((uint64_t)k << 32) | __float_as_uint(depth[r])) : 0ull;
    uint32_t p = pos - shift_out;
    const float4 co = conic_opacity[r];
    BinQ q;
    if (bin_prep(co.x, co.y, co.z, color_tau[r].w, q))
      bin_union(g, q, means2d + (size_t)r * g.C, [&](int t) {
        kdst[p] = kWide ? (KeyT)(((uint64_t)t << shift) | lo)
                        : (KeyT)(((uint32_t)t << shift) | g.key_code | k);
        vdst[p] = i;
        ++p;
      });
  }
  // The other items' tile rows are dealt out to the lanes, 32 units at a
  // time in (item, row) order. A unit's first list position is its item's
  // plus the pairs of the item's earlier rows: with R(u) the pairs of all the
  // warp's units before u (a running scan over the rounds) and Rb_j those of
  // item j's first unit (a scan of the counts over the lanes), it is
  // pos_j + R(u) - Rb_j.
  const bool units_here = in && n && !redo;
  const int units = units_here ? (int)((h >> 32) & 0xffull) : 0;
  int U, NU;
  const int ubase = warp_exclusive(units, lane, &U);
  const uint32_t rbase = (uint32_t)warp_exclusive(units_here ? (int)n : 0, lane, &NU);
  // this lane's item: cluster, Gaussian, and the depth half of a 64-bit key
  const uint32_t k_l = in ? r / (uint32_t)M : 0u;  // K M < 2^32
  const uint32_t i_l = in ? (uint32_t)(r - (uint64_t)k_l * M) : 0u;
  const uint32_t d_l = (kWide && units_here) ? __float_as_uint(depth[r]) : 0u;
  const int64_t s0w = s - lane;  // the warp's first item
  uint32_t carry = 0;
  // unit u: owner lane j, row rr of its item, row mask (the next round's
  // mask is fetched before this round's pairs are written)
  auto unit_at = [&](int u, int& j, int& rr, unsigned long long& mask) {
    j = unit_owner(ubase, u);
    rr = u - __shfl_sync(0xffffffffu, ubase, j);
    mask = u < U ? desc[s0w + j].mask[rr] : 0ull;
  };
  int j_nx = 0, rr_nx = 0;
  unsigned long long mask_nx = 0ull;
  if (U > 0) unit_at(lane, j_nx, rr_nx, mask_nx);
  for (int b = 0; b < U; b += 32) {
    const int j = j_nx, rr = rr_nx;
    const unsigned long long mask = mask_nx;
    if (b + 32 < U) unit_at(b + 32 + lane, j_nx, rr_nx, mask_nx);
    const unsigned long long hj = __shfl_sync(0xffffffffu, h, j);
    const uint32_t c = (uint32_t)__popcll(mask);
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    uint32_t p = __shfl_sync(0xffffffffu, pos, j) - shift_out + carry + (incl - c) -
                 __shfl_sync(0xffffffffu, rbase, j);
    carry += __shfl_sync(0xffffffffu, incl, 31);
    const uint32_t k = __shfl_sync(0xffffffffu, k_l, j);
    const uint32_t i = __shfl_sync(0xffffffffu, i_l, j);
    const uint64_t lo = kWide ? (((uint64_t)k << 32) | __shfl_sync(0xffffffffu, d_l, j)) : 0ull;
    const int ty0 = (int)(hj & 0xffffull), c0 = (int)((hj >> 16) & 0xffffull);
    unsigned long long m = mask;
    while (m) {
      const int bit = __ffsll((long long)m) - 1;
      m &= m - 1ull;
      const uint32_t t = (uint32_t)((ty0 + rr) * g.TX + c0 + bit);
      kdst[p] = kWide ? (KeyT)(((uint64_t)t << shift) | lo) : (KeyT)((t << shift) | g.key_code | k);
      vdst[p] = i;
      ++p;
    }
  }
  if (staged) {
    __syncwarp();
    for (uint32_t q = lane; q < total; q += 32) {
      keys[wbase + q] = s_key[warp][q];
      vals[wbase + q] = s_val[warp][q];
    }
  }
}

template <typename KeyT>
__global__ void __launch_bounds__(32 * kEmitWarps)
    k_bin_emit_staged(PanelGeom g, int64_t M, const float2* __restrict__ means2d,
                      const float4* __restrict__ conic_opacity, const float4* __restrict__ color_tau,
                      const float* __restrict__ depth, const uint32_t* __restrict__ order,
                      int64_t n_items, const uint32_t* __restrict__ counts,
                      const uint32_t* __restrict__ offsets, KeyT* __restrict__ keys,
                      uint32_t* __restrict__ vals, const BinDesc* __restrict__ desc,
                      const unsigned long long* __restrict__ P_dev, unsigned long long P_cap,
                      uint32_t* __restrict__ err) {
  bin_emit_block<KeyT>(g, M, means2d, conic_opacity, color_tau, depth, order, n_items, counts,
                       offsets, keys, vals, desc, P_dev, P_cap, err, blockIdx.x);
}

// The emit pass of every scene of a batch in one launch (32-bit pair keys);
// counts, offsets and descriptors indexed by batch position, order by scene
// position (scene-local item indices).
__global__ void __launch_bounds__(32 * kEmitWarps)
    k_bin_emit_batch(BatchBins bb, const uint32_t* __restrict__ order,
                     const uint32_t* __restrict__ counts, const uint32_t* __restrict__ offsets,
                     uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                     const BinDesc* __restrict__ desc, const unsigned long long* __restrict__ P_dev,
                     unsigned long long P_cap, uint32_t* __restrict__ err) {
  const SceneBins& sc = bb.sc[scene_of_block(bb, blockIdx.x)];
  bin_emit_block<uint32_t>(sc.g, sc.M, reinterpret_cast<const float2*>(sc.means2d),
                           reinterpret_cast<const float4*>(sc.conic_opacity),
                           reinterpret_cast<const float4*>(sc.color_tau), sc.depth, order + sc.off,
                           sc.n, counts + sc.off, offsets + sc.off, keys, vals, desc + sc.off, P_dev,
                           P_cap, err, blockIdx.x - sc.blk_off);
}

// Item keys of every scene of a batch: item p of the batch arrays is item
// p - off of its scene (keys with the scene's global clusters, values local).
__global__ void k_item_keys_batch(BatchBins bb, int64_t n_total, uint64_t* __restrict__ keys,
                                  uint32_t* __restrict__ vals) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_total) return;
  int s = 0;
  while (s + 1 < bb.n_scenes && p >= bb.sc[s + 1].off) ++s;
  const SceneBins& sc = bb.sc[s];
  const int64_t r = p - sc.off;
  const uint64_t k = (uint64_t)((uint32_t)r / (uint32_t)sc.M);
  const float tau = reinterpret_cast<const float4*>(sc.color_tau)[r].w;
  const uint32_t d = tau >= 0.f ? __float_as_uint(sc.depth[r]) : 0xffffffffu;
  keys[p] = ((k + (uint64_t)sc.g.cluster_base) << 32) | d;
  vals[p] = (uint32_t)r;
}

// Per scene, inv[off + perm[p]] = p - off for the scene's batch positions p.
__global__ void k_invert_batch(BatchBins bb, int64_t n_total, const uint32_t* __restrict__ perm,
                               uint32_t* __restrict__ inv) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_total) return;
  int s = 0;
  while (s + 1 < bb.n_scenes && p >= bb.sc[s + 1].off) ++s;
  const int64_t off = bb.sc[s].off;
  inv[off + perm[p]] = (uint32_t)(p - off);
}

__global__ void k_gather_u32(const uint32_t* __restrict__ src, const uint32_t* __restrict__ idx,
                             int64_t n, uint32_t* __restrict__ dst) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) dst[s] = src[idx[s]];
}

__global__ void k_invert_u32(const uint32_t* __restrict__ perm, int64_t n, uint32_t* __restrict__ inv) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) inv[perm[s]] = (uint32_t)s;
}

// One thread per (tile, cluster) run: lower bounds of its key and of the
// next key in the sorted pairs (the keys' upper 32 bits in Eq. 11 mode).
__global__ void k_ranges(PanelGeom g, int64_t P_cap, const unsigned long long* __restrict__ P_dev,
                         const uint32_t* __restrict__ keys32, const uint64_t* __restrict__ keys64,
                         uint2* __restrict__ ranges) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)g.T * g.K) return;
  int64_t P = P_cap;
  if (P_dev && *P_dev < (unsigned long long)P_cap) P = (int64_t)*P_dev;
  const int t = (int)(q / g.K), k = (int)(q - (int64_t)t * g.K);
  const uint32_t target = ((uint32_t)t << g.bit_k) | (uint32_t)k;
  auto tk_at = [&](int64_t i) -> uint32_t {
    return keys64 ? (uint32_t)(keys64[i] >> 32) : keys32[i];
  };
  int64_t lo = 0, hi = P;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (tk_at(mid) < target) lo = mid + 1;
    else hi = mid;
  }
  int64_t lo2 = lo;
  hi = P;
  while (lo2 < hi) {
    const int64_t mid = (lo2 + hi) >> 1;
    if (tk_at(mid) <= target) lo2 = mid + 1;
    else hi = mid;
  }
  ranges[q] = lo2 > lo ? make_uint2((uint32_t)lo, (uint32_t)lo2) : make_uint2(0u, 0u);
}

// Batched range table: one thread per (scene, tile, cluster).
__global__ void k_ranges_batch(BatchRangeArgs ra, int64_t P_cap, const unsigned long long* __restrict__ P_dev,
                               const uint32_t* __restrict__ keys32, uint2* __restrict__ ranges) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per_scene = (int64_t)ra.T_max * ra.K_glob;
  if (q >= per_scene * ra.n_scenes) return;
  const int sc = (int)(q / per_scene);
  const int64_t rem = q - (int64_t)sc * per_scene;
  const int t = (int)(rem / ra.K_glob), k = (int)(rem - (int64_t)t * ra.K_glob);
  if (t >= ra.T[sc] || k >= ra.K[sc]) {
    ranges[q] = make_uint2(0u, 0u);
    return;
  }
  int64_t P = P_cap;
  if (P_dev && *P_dev < (unsigned long long)P_cap) P = (int64_t)*P_dev;
  const uint32_t target = ((uint32_t)t << ra.bit_k) | ((uint32_t)sc << ra.bit_kc) | (uint32_t)k;
  int64_t lo = 0, hi = P;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (keys32[mid] < target) lo = mid + 1;
    else hi = mid;
  }
  int64_t lo2 = lo;
  hi = P;
  while (lo2 < hi) {
    const int64_t mid = (lo2 + hi) >> 1;
    if (keys32[mid] <= target) lo2 = mid + 1;
    else hi = mid;
  }
  ranges[q] = lo2 > lo ? make_uint2((uint32_t)lo, (uint32_t)lo2) : make_uint2(0u, 0u);
}

inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

cudaError_t launch_item_keys(const PanelGeom& g, int64_t M, const float* depth,
                             const float* color_tau, uint64_t* keys, uint32_t* vals,
                             cudaStream_t s) {
  const int64_t n = (int64_t)g.K * M;
  if (n == 0) return cudaSuccess;
  k_item_keys<<<blocks_for(n, 256), 256, 0, s>>>(g, M, depth,
                                                  reinterpret_cast<const float4*>(color_tau), keys,
                                                  vals);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_bin_count(const PanelGeom& g, int64_t M, const float* means2d,
                             const float* conic_opacity, const float* color_tau,
                             const uint32_t* order, const uint32_t* dest, int64_t n_items,
                             uint32_t* counts, void* desc, cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  const size_t smem = (size_t)kBoxFields * g.C * 32 * kBinWarps * sizeof(float);
  // the 48 KB default covers static and dynamic shared memory together (the
  // kernel's static part is its per-warp counters)
  if (smem + sizeof(uint32_t) * 32 * kBinWarps > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_bin_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_bin_count<<<blocks_for(n_items, 32 * kBinWarps), 32 * kBinWarps, smem, s>>>(
      g, M, reinterpret_cast<const float2*>(means2d),
      reinterpret_cast<const float4*>(conic_opacity), reinterpret_cast<const float4*>(color_tau),
      order, dest, n_items, counts, reinterpret_cast<BinDesc*>(desc));
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_bin_emit(const PanelGeom& g, int64_t M, const float* means2d,
                            const float* conic_opacity, const float* color_tau,
                            const float* depth, const uint32_t* order, int64_t n_items,
                            const uint32_t* offsets, uint32_t* keys32, uint64_t* keys64,
                            uint32_t* vals, const void* desc, cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  k_bin_emit<<<blocks_for(n_items, 128), 128, 0, s>>>(
      g, M, reinterpret_cast<const float2*>(means2d),
      reinterpret_cast<const float4*>(conic_opacity), reinterpret_cast<const float4*>(color_tau),
      depth, order, n_items, offsets, keys32, keys64, vals, reinterpret_cast<const BinDesc*>(desc));
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_bin_emit_coop(const PanelGeom& g, int64_t M, const float* means2d,
                                 const float* conic_opacity, const float* color_tau,
                                 const float* depth, const uint32_t* order, int64_t n_items,
                                 const uint32_t* counts, const uint32_t* offsets, uint32_t* keys32,
                                 uint64_t* keys64, uint32_t* vals, const void* desc,
                                 const unsigned long long* P_dev, unsigned long long P_cap,
                                 uint32_t* err, cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  const unsigned blocks = blocks_for(n_items, 32 * kEmitWarps);
  if (keys64)
    k_bin_emit_staged<uint64_t><<<blocks, 32 * kEmitWarps, 0, s>>>(
        g, M, reinterpret_cast<const float2*>(means2d),
        reinterpret_cast<const float4*>(conic_opacity), reinterpret_cast<const float4*>(color_tau),
        depth, order, n_items, counts, offsets, keys64, vals,
        reinterpret_cast<const BinDesc*>(desc), P_dev, P_cap, err);
  else
    k_bin_emit_staged<uint32_t><<<blocks, 32 * kEmitWarps, 0, s>>>(
        g, M, reinterpret_cast<const float2*>(means2d),
        reinterpret_cast<const float4*>(conic_opacity), reinterpret_cast<const float4*>(color_tau),
        depth, order, n_items, counts, offsets, keys32, vals,
        reinterpret_cast<const BinDesc*>(desc), P_dev, P_cap, err);
  note_launches(1);
  return cudaGetLastError();
}

// Block offsets of the scenes for a launch of `threads` items per block;
// returns the total block count.
inline uint32_t place_blocks(BatchBins& bb, int threads) {
  uint32_t b = 0;
  for (int i = 0; i < bb.n_scenes; ++i) {
    bb.sc[i].blk_off = b;
    b += (uint32_t)((bb.sc[i].n + threads - 1) / threads);
  }
  return b;
}

inline int64_t batch_items(const BatchBins& bb) {
  return bb.n_scenes ? bb.sc[bb.n_scenes - 1].off + bb.sc[bb.n_scenes - 1].n : 0;
}

cudaError_t launch_item_keys_batch(const BatchBins& bb, uint64_t* keys, uint32_t* vals, cudaStream_t s) {
  const int64_t n = batch_items(bb);
  if (n == 0) return cudaSuccess;
  k_item_keys_batch<<<blocks_for(n, 256), 256, 0, s>>>(bb, n, keys, vals);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_invert_batch(const BatchBins& bb, const uint32_t* perm, uint32_t* inv, cudaStream_t s) {
  const int64_t n = batch_items(bb);
  if (n == 0) return cudaSuccess;
  k_invert_batch<<<blocks_for(n, 256), 256, 0, s>>>(bb, n, perm, inv);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_bin_count_batch(const BatchBins& bb_in, const uint32_t* dest, uint32_t* counts, void* desc,
                                   cudaStream_t s) {
  BatchBins bb = bb_in;
  const uint32_t blocks = place_blocks(bb, 32 * kBinWarps);
  if (blocks == 0) return cudaSuccess;
  int C_max = 1;
  for (int i = 0; i < bb.n_scenes; ++i) C_max = max(C_max, bb.sc[i].g.C);
  const size_t smem = (size_t)kBoxFields * C_max * 32 * kBinWarps * sizeof(float);
  if (smem + sizeof(uint32_t) * 32 * kBinWarps > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_bin_count_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_bin_count_batch<<<blocks, 32 * kBinWarps, smem, s>>>(bb, dest, counts,
                                                         reinterpret_cast<BinDesc*>(desc));
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_bin_emit_batch(const BatchBins& bb_in, const uint32_t* order, const uint32_t* counts,
                                  const uint32_t* offsets, uint32_t* keys32, uint32_t* vals,
                                  const void* desc, const unsigned long long* P_dev,
                                  unsigned long long P_cap, uint32_t* err, cudaStream_t s) {
  BatchBins bb = bb_in;
  const uint32_t blocks = place_blocks(bb, 32 * kEmitWarps);
  if (blocks == 0) return cudaSuccess;
  k_bin_emit_batch<<<blocks, 32 * kEmitWarps, 0, s>>>(bb, order, counts, offsets, keys32, vals,
                                                      reinterpret_cast<const BinDesc*>(desc), P_dev,
                                                      P_cap, err);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_gather_u32(const uint32_t* src, const uint32_t* idx, int64_t n, uint32_t* dst,
                              cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_gather_u32<<<blocks_for(n, 256), 256, 0, s>>>(src, idx, n, dst);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_invert_u32(const uint32_t* perm, int64_t n, uint32_t* inv, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_invert_u32<<<blocks_for(n, 256), 256, 0, s>>>(perm, n, inv);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_ranges(const PanelGeom& g, int64_t P, const unsigned long long* P_dev,
                          const uint32_t* keys32, const uint64_t* keys64, uint2* ranges,
                          cudaStream_t s) {
  const int64_t runs = (int64_t)g.T * g.K;
  if (runs == 0) return cudaSuccess;
  k_ranges<<<blocks_for(runs, 256), 256, 0, s>>>(g, P, P_dev, keys32, keys64, ranges);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_ranges_batch(const BatchRangeArgs& r, int64_t P, const unsigned long long* P_dev,
                                const uint32_t* keys32, uint2* ranges, cudaStream_t s) {
  const int64_t n = (int64_t)r.n_scenes * r.T_max * r.K_glob;
  if (n == 0) return cudaSuccess;
  k_ranges_batch<<<blocks_for(n, 256), 256, 0, s>>>(r, P, P_dev, keys32, ranges);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace lfd
