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
__device__ __forceinline__ bool bin_row(const BinQ& g, const BinV& v, int ty, int TW, int TH,
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
  tx0 = (int)fx0 / TW;
  tx1 = (int)fx1 / TW;
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
    ty0 = min(ty0, v.y0 / pg.TH);
    ty1 = max(ty1, v.y1 / pg.TH);
    c0 = min(c0, (int)v.bx0 / pg.TW);
    c1 = max(c1, (int)v.bx1 / pg.TW);
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
        if (!bin_row(q, v, ty, pg.TW, pg.TH, a, b)) continue;
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
constexpr int kDescRows = 7;
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
  const uint64_t k = (uint64_t)(r / M);
  const float tau = color_tau[r].w;
  const uint32_t d = tau >= 0.f ? __float_as_uint(depth[r]) : 0xffffffffu;
  keys[r] = (k << 32) | d;
  vals[r] = (uint32_t)r;
}

__global__ void k_bin_count(PanelGeom g, int64_t M, const float2* __restrict__ means2d,
                            const float4* __restrict__ conic_opacity,
                            const float4* __restrict__ color_tau, const uint32_t* __restrict__ order,
                            int64_t n_items, uint32_t* __restrict__ counts,
                            BinDesc* __restrict__ desc) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_items) return;
  const uint32_t r = order ? order[s] : (uint32_t)s;
  const float4 co = conic_opacity[r];
  BinQ q;
  uint32_t n = 0;
  unsigned long long header = 0ull;
  if (bin_prep(co.x, co.y, co.z, color_tau[r].w, q)) {
    const float2* means = means2d + (size_t)r * g.C;
    int ty0, ty1, c0, c1;
    bin_extent(g, q, means, ty0, ty1, c0, c1);
    const int rows = ty1 >= ty0 ? ty1 - ty0 + 1 : 0;
    const bool fits = rows <= kDescRows && (rows == 0 || c1 - c0 < 64);
    n = bin_rows(g, q, means, ty0, ty1, c0, c1, [&](int ty, int, unsigned long long mask) {
      if (desc && fits) desc[s].mask[ty - ty0] = mask;
    });
    header = rows == 0 ? 0ull
                       : ((unsigned long long)ty0 | ((unsigned long long)c0 << 16) |
                          ((unsigned long long)rows << 32) | ((unsigned long long)(fits ? 0 : 1) << 40));
  }
  counts[s] = n;
  if (desc) desc[s].header = header;
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
  const uint32_t k = (uint32_t)(r / M);
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

__global__ void k_ranges(PanelGeom g, int64_t P, const uint32_t* __restrict__ keys32,
                         const uint64_t* __restrict__ keys64, uint2* __restrict__ ranges) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  auto tk_at = [&](int64_t q) -> uint32_t {
    return keys64 ? (uint32_t)(keys64[q] >> 32) : keys32[q];
  };
  const uint32_t tk = tk_at(p);
  const uint32_t t = tk >> g.bit_k;
  const uint32_t k = tk & ((1u << g.bit_k) - 1u);
  uint2* r = ranges + (size_t)t * g.K + k;
  if (p == 0 || tk_at(p - 1) != tk) r->x = (uint32_t)p;
  if (p == P - 1 || tk_at(p + 1) != tk) r->y = (uint32_t)(p + 1);
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
                             const uint32_t* order, int64_t n_items, uint32_t* counts, void* desc,
                             cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  k_bin_count<<<blocks_for(n_items, 128), 128, 0, s>>>(
      g, M, reinterpret_cast<const float2*>(means2d),
      reinterpret_cast<const float4*>(conic_opacity), reinterpret_cast<const float4*>(color_tau),
      order, n_items, counts, reinterpret_cast<BinDesc*>(desc));
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

cudaError_t launch_ranges(const PanelGeom& g, int64_t P, const uint32_t* keys32,
                          const uint64_t* keys64, uint2* ranges, cudaStream_t s) {
  if (P == 0) return cudaSuccess;
  k_ranges<<<blocks_for(P, 256), 256, 0, s>>>(g, P, keys32, keys64, ranges);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace lfd
