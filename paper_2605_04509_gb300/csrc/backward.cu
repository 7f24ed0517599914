// Backward pass of the interlaced render: gradients of a loss of the image
// with respect to the Gaussians' means, scales, rotations, opacities and SH
// coefficients. Not in the paper; it differentiates the same definitions
// (Eq. 5-6 projection with attribute reuse, Eq. 9-10 blend with the 3DGS
// rules). No per-subpixel lists are stored by the forward pass. Each
// subpixel needs its final transmittance and the list entry where it
// stopped: the forward keeps those 8 bytes per subpixel when asked
// (LFD_FLAG_KEEP_BLEND_STATE), otherwise the subpixel re-blends its
// (tile, cluster) list front to back to find them. It then walks the list
// back to front.
#include "lfd_internal.h"

namespace lfd {
namespace {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;

// Sum NV values (a power of two up to 32) over a warp with NV - 1 + 5 -
// log2(NV) shuffles: each butterfly stage trades half of the values still
// held with the partner lane, so lane l ends with the full sum of
// v[l >> (5 - log2(NV))] (v is overwritten). All 32 lanes must call it.
template <int NV>
__device__ __forceinline__ float warp_transpose_sum(float (&v)[NV], int lane) {
  const unsigned full = 0xffffffffu;
  int off = 16;
#pragma unroll
  for (int half = NV / 2; half >= 1; half >>= 1, off >>= 1) {
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float send = up ? v[i] : v[i + half];
      const float keep = up ? v[i + half] : v[i];
      v[i] = keep + __shfl_xor_sync(full, send, off);
    }
  }
  float r = v[0];
#pragma unroll
  for (; off >= 1; off >>= 1) r += __shfl_xor_sync(full, r, off);
  return r;
}

// ---------------------------------------------------------------------------
// blend backward: one CTA per (tile, cluster) run of Psi, one subpixel per
// thread. Each subpixel needs its final transmittance and the list position
// where its walk stopped: KEPT reads them from the forward frame, otherwise
// the list is re-blended front to back (the forward blend's arithmetic,
// staged batch by batch in shared memory). The list is then staged again
// from the last needed batch back to the first and walked back to front.
// As in the forward blend, each staged entry gets a bit per cluster view
// telling whether that view's region (bounding box, one pixel of margin)
// meets the tile; a subpixel only evaluates entries with its view's bit (the
// others have alpha < 1/255 there). Psi lists a run's subpixels view by
// view, so a warp holds one or two views: it walks the entries seen by any
// of them, all lanes on the same entry, and sums each entry's gradients over
// the warp (16-value transpose reduction). Conic, opacity and colour sums
// collect in shared memory and go to global memory once per entry and batch,
// by the thread that staged the entry; mean sums go to global memory at once.
// ---------------------------------------------------------------------------
template <bool KEPT>
__global__ void __launch_bounds__(256) k_blend_backward(PanelGeom g, BlendArgs a, BlendGrads gr) {
  extern __shared__ float4 smem[];
  const int NB = blockDim.x;
  const int NW = NB >> 5;
  const int C = g.C;
  float4* s_co = smem;                                          // raw conic (a, b, c), opacity
  float4* s_col = smem + NB;                                    // colour
  float4* s_gco = smem + 2 * NB;                                // d(a, b, c), d opacity
  float4* s_gcol = smem + 3 * NB;                               // d colour
  float2* s_mean = reinterpret_cast<float2*>(smem + 4 * NB);    // [C][NB]
  uint32_t* s_gid = reinterpret_cast<uint32_t*>(s_mean + C * NB);
  uint32_t* s_vm = s_gid + NB;                                  // view bits of each entry
  // per-view lists of the re-blend (without KEPT only)
  uint16_t* s_idx = reinterpret_cast<uint16_t*>(s_vm + NB);     // [C][NB]
  int* s_cnt = reinterpret_cast<int*>(s_idx + ((C * NB + 1) & ~1));  // [C][NW + 1]
  __shared__ uint32_t s_last;
  const int k = blockIdx.x / g.T;
  const int t = blockIdx.x - k * g.T;
  const int s0 = a.seg[(size_t)t * (g.K + 1) + k];
  const int n = a.seg[(size_t)t * (g.K + 1) + k + 1] - s0;
  if (n <= 0) return;
  const uint2 rg = a.ranges[(size_t)t * g.K + k];
  if (rg.x == rg.y) return;
  const int tx = t % g.TX, ty = t / g.TX;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const float bx0 = (float)(tx * g.TW) + 0.5f - 1.f;
  const float bx1 = (float)min(tx * g.TW + g.TW, g.W) - 0.5f + 1.f;
  const float by0 = (float)(ty * g.TH) + 0.5f - 1.f;
  const float by1 = (float)min(ty * g.TH + g.TH, g.H) - 0.5f + 1.f;

  // stage entry base + threadIdx.x: attributes, means and view bits; with
  // compact, also list per view the staged entries with that view's bit.
  // Called by every thread; it synchronises the block.
  auto stage = [&](uint32_t base, bool compact) {
    const uint32_t e = base + threadIdx.x;
    uint32_t mask = 0;
    if (e < rg.y) {
      const uint32_t gid = a.list[e];
      const size_t rec = (size_t)k * a.M + gid;
      const float4 co = reinterpret_cast<const float4*>(a.conic_opacity)[rec];
      const float4 ct = reinterpret_cast<const float4*>(a.color_tau)[rec];
      s_co[threadIdx.x] = co;
      s_col[threadIdx.x] = ct;
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
      s_gid[threadIdx.x] = gid;
    }
    s_vm[threadIdx.x] = mask;
    if (!compact) {
      __syncthreads();
      return;
    }
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
      if ((mask >> l) & 1u)
        s_idx[l * NB + s_cnt[l * (NW + 1) + warp] + __popc(b & lt)] = (uint16_t)threadIdx.x;
    }
    __syncthreads();
  };
  // add the staged entry's shared-memory sums (conic, opacity and colour
  // gradients) to global memory (entry base + threadIdx.x, by the thread
  // that staged it) and clear them
  auto flush = [&](uint32_t base, uint32_t end) {
    const uint32_t e = base + threadIdx.x;
    if (e < end && s_vm[threadIdx.x]) {
      const uint32_t gid = s_gid[threadIdx.x];
      const size_t rec = (size_t)k * a.M + gid;
      const float4 d = s_gco[threadIdx.x];
      if (d.x != 0.f) atomicAdd(&gr.grad_conic[4 * rec + 0], d.x);
      if (d.y != 0.f) atomicAdd(&gr.grad_conic[4 * rec + 1], d.y);
      if (d.z != 0.f) atomicAdd(&gr.grad_conic[4 * rec + 2], d.z);
      if (d.w != 0.f) atomicAdd(&gr.grad_opac[gid], d.w);
      const float4 dc = s_gcol[threadIdx.x];
      if (dc.x != 0.f) atomicAdd(&gr.grad_color[4 * rec + 0], dc.x);
      if (dc.y != 0.f) atomicAdd(&gr.grad_color[4 * rec + 1], dc.y);
      if (dc.z != 0.f) atomicAdd(&gr.grad_color[4 * rec + 2], dc.z);
    }
    s_gco[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
    s_gcol[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
  };

  // runs longer than the block are processed in chunks of blockDim subpixels
  for (int chunk = 0; chunk < n; chunk += NB) {
    const int r = chunk + threadIdx.x;
    const bool live = r < n;
    float px = 0.f, py = 0.f, G = 0.f;
    int slot = 0, ch = 0;
    if (live) {
      const uint32_t e = a.psi[(size_t)t * g.cap + s0 + r];
      const int view = (int)(e >> 16);
      const int loc = (int)(e & 0xffffu);
      const int xl = (loc / 3) % g.TW, yl = (loc / 3) / g.TW;
      const int x = tx * g.TW + xl, y = ty * g.TH + yl;
      ch = loc % 3;
      px = (float)x + 0.5f;
      py = (float)y + 0.5f;
      slot = view - k * C;
      G = gr.grad_out[((int64_t)y * g.W + x) * 3 + ch];
    }
    // the opacity of an entry for this subpixel, exactly as the forward
    // blend computes it (0 when skipped); also e^power and whether clamped
    auto opacity_of = [&](int gi, float& vexp, bool& clamped) -> float {
      const float4 co = s_co[gi];
      const float2 mu = s_mean[slot * NB + gi];
      const float dx = px - mu.x, dy = py - mu.y;
      // the forward blend's pre-scaled conic and order of operations
      const float power = quad_power(-0.5f * kLog2e * co.x, -kLog2e * co.y, -0.5f * kLog2e * co.z, dx, dy);
      if (power > 0.f) return 0.f;
      const float ev = ex2_approx(power);
      const float v = co.w * ev;
      if (!(v >= kAlphaMin)) return 0.f;
      vexp = ev;
      clamped = v > kAlphaMax;
      return fminf(kAlphaMax, v);
    };

    // final transmittance and the list index of the first entry not added
    float T = 1.f;
    uint32_t last = rg.x;
    if (KEPT) {
      if (live) {
        const uint2 kp = a.keep[(size_t)t * g.cap + s0 + r];
        last = kp.x;
        T = __uint_as_float(kp.y);
      }
    } else {
      bool act = live;
      uint32_t stop = rg.y;
      for (uint32_t base = rg.x; base < rg.y; base += (uint32_t)NB) {
        if (!__syncthreads_or(act)) break;
        stage(base, true);
        if (!act) continue;
        const uint16_t* idx = s_idx + slot * NB;
        const int cnt = s_cnt[slot * (NW + 1) + NW];
        for (int q = 0; q < cnt; ++q) {
          const int gi = idx[q];
          float ve;
          bool cl;
          const float alpha = opacity_of(gi, ve, cl);
          if (alpha == 0.f) continue;
          const float Tn = T * (1.f - alpha);
          if (Tn < kTMin) {
            act = false;
            stop = base + (uint32_t)gi;
            break;
          }
          T = Tn;
        }
      }
      if (live) last = stop;
    }
    // the block's furthest stop
    __syncthreads();
    if (threadIdx.x == 0) s_last = rg.x;
    __syncthreads();
    if (live) atomicMax(&s_last, last);
    __syncthreads();
    const uint32_t end = s_last;
    if (end == rg.x) continue;

    // back to front over [rg.x, last): R is the colour of everything behind.
    // Per entry, the warp sums its conic, opacity and colour gradients and
    // the mean gradients of its lowest view v0 and highest view v1 (16
    // slots, 12 used); the reducing lanes add the mean sums to global memory
    // directly (a view strictly between v0 and v1 adds its own).
    float R = ch == 0 ? a.bg[0] : (ch == 1 ? a.bg[1] : a.bg[2]);
    const unsigned wm = __reduce_or_sync(0xffffffffu, live ? (1u << slot) : 0u);
    const int v0 = wm ? __ffs(wm) - 1 : 0;
    const int v1 = wm ? 31 - __clz(wm) : 0;
    // the warp walks no entry at or past its furthest stop
    const uint32_t wlast = __reduce_max_sync(0xffffffffu, live ? last : rg.x);
    const uint32_t nb_total = (end - rg.x + NB - 1) / NB;
    s_gco[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
    s_gcol[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int b = (int)nb_total - 1; b >= 0; --b) {
      const uint32_t base = rg.x + (uint32_t)b * NB;
      // the thread that staged entry i of the batch behind flushes it before
      // staging entry i of this one: no barrier between the two
      if (b != (int)nb_total - 1) flush(base + (uint32_t)NB, end);
      stage(base, false);
      for (int w32 = NW - 1; wm != 0u && w32 >= 0; --w32) {
        const uint32_t e_lane = base + (uint32_t)(w32 * 32 + lane);
        unsigned h = __ballot_sync(0xffffffffu, e_lane < wlast && (s_vm[w32 * 32 + lane] & wm) != 0u);
        while (h) {
          const int j = 31 - __clz(h);
          h &= ~(1u << j);
          const int gi = w32 * 32 + j;
          float v[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = 0.f;
          bool any = false;
          if (live && base + (uint32_t)gi < last && ((s_vm[gi] >> slot) & 1u)) {
            float ve = 0.f;
            bool cl = false;
            const float alpha = opacity_of(gi, ve, cl);
            if (alpha != 0.f) {
              any = true;
              const float4 col4 = s_col[gi];
              const float c = ch == 0 ? col4.x : (ch == 1 ? col4.y : col4.z);
              const float Ti = __fdividef(T, 1.f - alpha);  // transmittance in front of this entry
              const float dcol = alpha * Ti * G;
              v[4] = ch == 0 ? dcol : 0.f;
              v[5] = ch == 1 ? dcol : 0.f;
              v[6] = ch == 2 ? dcol : 0.f;
              const float dalpha = (c - R) * Ti * G;
              R = c * alpha + (1.f - alpha) * R;
              T = Ti;
              if (!cl) {
                const float4 co = s_co[gi];
                const float2 mu = s_mean[slot * NB + gi];
                const float dx = px - mu.x, dy = py - mu.y;
                const float dpower = dalpha * alpha;  // d alpha / d power = alpha
                // power = -(a dx^2 + 2 b dx dy + c dy^2) / 2, dx = px - mu_x
                v[0] = -0.5f * dpower * dx * dx;
                v[1] = -dpower * dx * dy;
                v[2] = -0.5f * dpower * dy * dy;
                v[3] = dalpha * ve;
                const float dmx = dpower * (co.x * dx + co.y * dy);
                const float dmy = dpower * (co.y * dx + co.z * dy);
                if (slot == v0) {
                  v[8] = dmx;
                  v[9] = dmy;
                } else if (slot == v1) {
                  v[10] = dmx;
                  v[11] = dmy;
                } else {
                  float* gm = gr.grad_means2d + 2 * (((size_t)k * a.M + s_gid[gi]) * C + slot);
                  atomicAdd(gm + 0, dmx);
                  atomicAdd(gm + 1, dmy);
                }
              }
            }
          }
          if (!__any_sync(0xffffffffu, any)) continue;
          // lanes 2i and 2i + 1 end with the warp's sum of v[i] (v[7] unused)
          const float sum = warp_transpose_sum<16>(v, lane);
          const int i = lane >> 1;
          if ((lane & 1) == 0 && i < 12 && sum != 0.f) {
            if (i < 4) {
              atomicAdd(reinterpret_cast<float*>(&s_gco[gi]) + i, sum);
            } else if (i < 7) {
              atomicAdd(reinterpret_cast<float*>(&s_gcol[gi]) + (i - 4), sum);
            } else if (i >= 8) {
              const int vv = i < 10 ? v0 : v1;
              atomicAdd(gr.grad_means2d + 2 * (((size_t)k * a.M + s_gid[gi]) * C + vv) + (i & 1), sum);
            }
          }
        }
      }
      __syncthreads();
    }
    flush(rg.x, end);
  }
}

// ---------------------------------------------------------------------------
// projection backward: one thread per Gaussian, every cluster and slot
// ---------------------------------------------------------------------------
__device__ __forceinline__ float3 cam_point(const float* c, float x, float y, float z) {
  return make_float3(c[0] * x + c[1] * y + c[2] * z + c[9], c[3] * x + c[4] * y + c[5] * z + c[10],
                     c[6] * x + c[7] * y + c[8] * z + c[11]);
}

constexpr float kC0 = 0.28209479177387814f;
constexpr float kC1 = 0.4886025119029199f;
constexpr float kC2a = 1.0925484305920792f;
constexpr float kC2b = 0.31539156525252005f;
constexpr float kC2c = 0.5462742152960396f;
constexpr float kC3a = 0.5900435899266435f;
constexpr float kC3b = 2.890611442640554f;
constexpr float kC3c = 0.4570457994644658f;
constexpr float kC3d = 0.3731763325901154f;
constexpr float kC3e = 1.445305721320277f;

__global__ void __launch_bounds__(128) k_project_backward(PanelGeom g, CamTable cams, ProjectArgs a,
                                                          BlendGrads gr, ParamGrads out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.M) return;
  const float* means = a.means;
  const float* scales = reinterpret_cast<const float*>(a.scales);
  const float* quats = reinterpret_cast<const float*>(a.quats);
  const float* shs = reinterpret_cast<const float*>(a.sh);
  const float mx = means[3 * i], my = means[3 * i + 1], mz = means[3 * i + 2];
  const float qr[4] = {quats[4 * i], quats[4 * i + 1], quats[4 * i + 2], quats[4 * i + 3]};
  const float sx = scales[3 * i], sy = scales[3 * i + 1], sz = scales[3 * i + 2];
  const int ncoef = (a.sh_degree + 1) * (a.sh_degree + 1);

  const float qn = rsqrtf(qr[0] * qr[0] + qr[1] * qr[1] + qr[2] * qr[2] + qr[3] * qr[3]);
  const float qw = qr[0] * qn, qx = qr[1] * qn, qy = qr[2] * qn, qz = qr[3] * qn;
  float Rq[3][3] = {{1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy)},
                    {2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx)},
                    {2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)}};
  const float s[3] = {sx, sy, sz};
  float Mm[3][3];  // Rq diag(s)
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) Mm[r][c] = Rq[r][c] * s[c];
  float S3[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) S3[r][c] = Mm[r][0] * Mm[c][0] + Mm[r][1] * Mm[c][1] + Mm[r][2] * Mm[c][2];

  float dmu[3] = {0.f, 0.f, 0.f};
  float dS3[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  // the SH record in registers (zero past the degree), loops over all 16
  // coefficients fully unrolled, so that nothing is indexed at run time
  float sh[16][3], dsh[16][3];
#pragma unroll
  for (int c = 0; c < 16; ++c)
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      sh[c][u] = c < ncoef ? shs[((size_t)i * ncoef + c) * 3 + u] : 0.f;
      dsh[c][u] = 0.f;
    }

  for (int k = 0; k < g.K; ++k) {
    const size_t rec = (size_t)k * a.M + i;
    // per-view means (Eq. 5)
    for (int l = 0; l < g.C; ++l) {
      const float gx = gr.grad_means2d[2 * (rec * g.C + l)];
      const float gy = gr.grad_means2d[2 * (rec * g.C + l) + 1];
      if (gx == 0.f && gy == 0.f) continue;
      const int j = min(k * g.C + l, g.N - 1);
      const float* cj = cams.c[j];
      const float3 p = cam_point(cj, mx, my, mz);
      const float iz = 1.f / p.z;
      const float dpx = cj[12] * iz * gx, dpy = cj[13] * iz * gy;
      const float dpz = -(cj[12] * p.x * gx + cj[13] * p.y * gy) * iz * iz;
      dmu[0] += cj[0] * dpx + cj[3] * dpy + cj[6] * dpz;
      dmu[1] += cj[1] * dpx + cj[4] * dpy + cj[7] * dpz;
      dmu[2] += cj[2] * dpx + cj[5] * dpy + cj[8] * dpz;
    }
    const float4 gcon = reinterpret_cast<const float4*>(gr.grad_conic)[rec];
    const float4 gcol = reinterpret_cast<const float4*>(gr.grad_color)[rec];
    const float4 ct = reinterpret_cast<const float4*>(a.color_tau)[rec];
    if (!(ct.w >= 0.f)) continue;  // culled for this cluster
    const int jr = min(k * g.C + g.C / 2, g.N - 1);
    const float* cr = cams.c[jr];
    const float3 p = cam_point(cr, mx, my, mz);
    // ---- colour (SH at the representative camera centre) ----
    if (gcol.x != 0.f || gcol.y != 0.f || gcol.z != 0.f) {
      const float cpx = -(cr[0] * cr[9] + cr[3] * cr[10] + cr[6] * cr[11]);
      const float cpy = -(cr[1] * cr[9] + cr[4] * cr[10] + cr[7] * cr[11]);
      const float cpz = -(cr[2] * cr[9] + cr[5] * cr[10] + cr[8] * cr[11]);
      const float ux = mx - cpx, uy = my - cpy, uz = mz - cpz;
      const float inv = rsqrtf(ux * ux + uy * uy + uz * uz);
      const float x = ux * inv, y = uy * inv, z = uz * inv;
      const float xx = x * x, yy = y * y, zz = z * z;
      const float b[16] = {kC0, -kC1 * y, kC1 * z, -kC1 * x, kC2a * x * y, -kC2a * y * z,
                           kC2b * (2.f * zz - xx - yy), -kC2a * x * z, kC2c * (xx - yy),
                           -kC3a * y * (3.f * xx - yy), kC3b * x * y * z, -kC3c * y * (4.f * zz - xx - yy),
                           kC3d * z * (2.f * zz - 3.f * xx - 3.f * yy), -kC3c * x * (4.f * zz - xx - yy),
                           kC3e * z * (xx - yy), -kC3a * x * (xx - 3.f * yy)};
      const float bx[16] = {0.f, 0.f, 0.f, -kC1, kC2a * y, 0.f, -2.f * kC2b * x, -kC2a * z, 2.f * kC2c * x,
                            -6.f * kC3a * x * y, kC3b * y * z, 2.f * kC3c * x * y, -6.f * kC3d * x * z,
                            -kC3c * (4.f * zz - 3.f * xx - yy), 2.f * kC3e * x * z, -kC3a * (3.f * xx - 3.f * yy)};
      const float by[16] = {0.f, -kC1, 0.f, 0.f, kC2a * x, -kC2a * z, -2.f * kC2b * y, 0.f, -2.f * kC2c * y,
                            -kC3a * (3.f * xx - 3.f * yy), kC3b * x * z, -kC3c * (4.f * zz - xx - 3.f * yy),
                            -6.f * kC3d * y * z, 2.f * kC3c * x * y, -2.f * kC3e * y * z, 6.f * kC3a * x * y};
      const float bz[16] = {0.f, 0.f, kC1, 0.f, 0.f, -kC2a * y, 4.f * kC2b * z, -kC2a * x, 0.f, 0.f,
                            kC3b * x * y, -8.f * kC3c * y * z, kC3d * (6.f * zz - 3.f * xx - 3.f * yy),
                            -8.f * kC3c * x * z, kC3e * (xx - yy), 0.f};
      const float gc[3] = {gcol.x, gcol.y, gcol.z};
      float ddx = 0.f, ddy = 0.f, ddz = 0.f;
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        float v = 0.5f;
#pragma unroll
        for (int c = 0; c < 16; ++c) v += b[c] * sh[c][u];
        if (!(v > 0.f)) continue;  // clamped at zero: no gradient
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          dsh[c][u] += b[c] * gc[u];
          const float sv = sh[c][u] * gc[u];
          ddx += bx[c] * sv;
          ddy += by[c] * sv;
          ddz += bz[c] * sv;
        }
      }
      // through the normalisation of the direction
      const float dot = x * ddx + y * ddy + z * ddz;
      dmu[0] += (ddx - x * dot) * inv;
      dmu[1] += (ddy - y * dot) * inv;
      dmu[2] += (ddz - z * dot) * inv;
    }
    // ---- covariance: conic -> Sigma2D -> (Sigma3D, Jacobian) ----
    if (gcon.x == 0.f && gcon.y == 0.f && gcon.z == 0.f) continue;
    const float fx = cr[12], fy = cr[13];
    const float limx = 1.3f * (0.5f * (float)g.W / fx);
    const float limy = 1.3f * (0.5f * (float)g.H / fy);
    const float iz = 1.f / p.z;
    const float rx = p.x * iz, ry = p.y * iz;
    const bool clx = rx < -limx || rx > limx, cly = ry < -limy || ry > limy;
    const float txz = fminf(fmaxf(rx, -limx), limx);
    const float tyz = fminf(fmaxf(ry, -limy), limy);
    const float J[2][3] = {{fx * iz, 0.f, -fx * txz * iz}, {0.f, fy * iz, -fy * tyz * iz}};
    float Tm[2][3];
    for (int r = 0; r < 2; ++r)
      for (int c = 0; c < 3; ++c) Tm[r][c] = J[r][0] * cr[c] + J[r][1] * cr[3 + c] + J[r][2] * cr[6 + c];
    float TS[2][3];  // Tm S3
    for (int r = 0; r < 2; ++r)
      for (int c = 0; c < 3; ++c) TS[r][c] = Tm[r][0] * S3[0][c] + Tm[r][1] * S3[1][c] + Tm[r][2] * S3[2][c];
    const float Sxx = TS[0][0] * Tm[0][0] + TS[0][1] * Tm[0][1] + TS[0][2] * Tm[0][2] + 0.3f;
    const float Sxy = TS[0][0] * Tm[1][0] + TS[0][1] * Tm[1][1] + TS[0][2] * Tm[1][2];
    const float Syy = TS[1][0] * Tm[1][0] + TS[1][1] * Tm[1][1] + TS[1][2] * Tm[1][2] + 0.3f;
    const float det = Sxx * Syy - Sxy * Sxy;
    const float id2 = 1.f / (det * det);
    // conic (a, b, c) = (Syy, -Sxy, Sxx) / det
    const float da = gcon.x, db = gcon.y, dc = gcon.z;
    const float dSxx = -Syy * Syy * id2 * da + Sxy * Syy * id2 * db + (1.f / det - Sxx * Syy * id2) * dc;
    const float dSyy = (1.f / det - Sxx * Syy * id2) * da + Sxy * Sxx * id2 * db - Sxx * Sxx * id2 * dc;
    const float dSxy = 2.f * Sxy * Syy * id2 * da + (-1.f / det - 2.f * Sxy * Sxy * id2) * db +
                       2.f * Sxy * Sxx * id2 * dc;
    // symmetric matrix gradient of Sigma2D
    const float Gm[2][2] = {{dSxx, 0.5f * dSxy}, {0.5f * dSxy, dSyy}};
    // dSigma3D += Tm^T G Tm
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c)
        dS3[r][c] += Tm[0][r] * (Gm[0][0] * Tm[0][c] + Gm[0][1] * Tm[1][c]) +
                     Tm[1][r] * (Gm[1][0] * Tm[0][c] + Gm[1][1] * Tm[1][c]);
    // dTm = 2 G Tm S3, dJ = dTm W^T
    float dTm[2][3];
    for (int r = 0; r < 2; ++r)
      for (int c = 0; c < 3; ++c) dTm[r][c] = 2.f * (Gm[r][0] * TS[0][c] + Gm[r][1] * TS[1][c]);
    float dJ[2][3];
    for (int r = 0; r < 2; ++r)
      for (int c = 0; c < 3; ++c) dJ[r][c] = dTm[r][0] * cr[3 * c] + dTm[r][1] * cr[3 * c + 1] + dTm[r][2] * cr[3 * c + 2];
    // J00 = fx/z, J02 = -fx txz / z, J11 = fy/z, J12 = -fy tyz / z
    float dpx = 0.f, dpy = 0.f, dpz = 0.f;
    dpz += dJ[0][0] * (-fx * iz * iz) + dJ[1][1] * (-fy * iz * iz);
    if (clx) {
      dpz += dJ[0][2] * (fx * txz * iz * iz);
    } else {
      dpx += dJ[0][2] * (-fx * iz * iz);
      dpz += dJ[0][2] * (2.f * fx * p.x * iz * iz * iz);
    }
    if (cly) {
      dpz += dJ[1][2] * (fy * tyz * iz * iz);
    } else {
      dpy += dJ[1][2] * (-fy * iz * iz);
      dpz += dJ[1][2] * (2.f * fy * p.y * iz * iz * iz);
    }
    dmu[0] += cr[0] * dpx + cr[3] * dpy + cr[6] * dpz;
    dmu[1] += cr[1] * dpx + cr[4] * dpy + cr[7] * dpz;
    dmu[2] += cr[2] * dpx + cr[5] * dpy + cr[8] * dpz;
  }
  // Sigma3D = Mm Mm^T -> dMm = 2 dS3_sym Mm (dS3 is accumulated symmetric)
  float dM[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      dM[r][c] = (dS3[r][0] + dS3[0][r]) * Mm[0][c] + (dS3[r][1] + dS3[1][r]) * Mm[1][c] +
                 (dS3[r][2] + dS3[2][r]) * Mm[2][c];
  float dR[3][3];
  float ds[3] = {0.f, 0.f, 0.f};
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      dR[r][c] = dM[r][c] * s[c];
      ds[c] += dM[r][c] * Rq[r][c];
    }
  const float dw = 2.f * (-qz * dR[0][1] + qy * dR[0][2] + qz * dR[1][0] - qx * dR[1][2] - qy * dR[2][0] + qx * dR[2][1]);
  const float dxq = 2.f * (qy * dR[0][1] + qz * dR[0][2] + qy * dR[1][0] - 2.f * qx * dR[1][1] - qw * dR[1][2] +
                           qz * dR[2][0] + qw * dR[2][1] - 2.f * qx * dR[2][2]);
  const float dyq = 2.f * (-2.f * qy * dR[0][0] + qx * dR[0][1] + qw * dR[0][2] + qx * dR[1][0] + qz * dR[1][2] -
                           qw * dR[2][0] + qz * dR[2][1] - 2.f * qy * dR[2][2]);
  const float dzq = 2.f * (-2.f * qz * dR[0][0] - qw * dR[0][1] + qx * dR[0][2] + qw * dR[1][0] - 2.f * qz * dR[1][1] +
                           qy * dR[1][2] + qx * dR[2][0] + qy * dR[2][1]);
  const float dqn[4] = {dw, dxq, dyq, dzq};
  const float qv[4] = {qw, qx, qy, qz};
  const float dd = qv[0] * dqn[0] + qv[1] * dqn[1] + qv[2] * dqn[2] + qv[3] * dqn[3];
  for (int c = 0; c < 4; ++c) out.quats[4 * i + c] = (dqn[c] - qv[c] * dd) * qn;
  for (int c = 0; c < 3; ++c) {
    out.means[3 * i + c] = dmu[c];
    out.scales[3 * i + c] = ds[c];
  }
  out.opacities[i] = gr.grad_opac[i];
#pragma unroll
  for (int c = 0; c < 16; ++c)
#pragma unroll
    for (int u = 0; u < 3; ++u)
      if (c < ncoef) out.sh[((size_t)i * ncoef + c) * 3 + u] = dsh[c][u];
}

}  // namespace

cudaError_t launch_blend_backward(const PanelGeom& g, const BlendArgs& a, const BlendGrads& gr,
                                  cudaStream_t s) {
  if ((int64_t)g.K * g.T == 0) return cudaSuccess;
  const int need = a.max_segment > 0 ? a.max_segment : 1;
  // 128 threads: a run of more subpixels is taken in chunks, each staging
  // the list again, but fewer warps wait at each batch's barriers for the
  // slowest one (256-thread blocks were 7 % slower on 256-subpixel runs)
  const int block = min(128, ((need + 31) / 32) * 32);
  const int nw = block / 32;
  // the per-view lists are only needed to re-blend (no kept state)
  const size_t smem = (size_t)block * (4 * sizeof(float4) + g.C * sizeof(float2) + 2 * sizeof(uint32_t)) +
                      (a.keep ? 0 : (((size_t)g.C * block + 1) & ~(size_t)1) * sizeof(uint16_t) +
                                        (size_t)g.C * (nw + 1) * sizeof(int));
  const unsigned grid = (unsigned)((int64_t)g.K * g.T);
  // the 48 KB default covers the kernel's static word as well
  const bool big = smem + 16 > 48 * 1024;
  if (a.keep) {
    if (big)
      cudaFuncSetAttribute(k_blend_backward<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_blend_backward<true><<<grid, block, smem, s>>>(g, a, gr);
  } else {
    if (big)
      cudaFuncSetAttribute(k_blend_backward<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_blend_backward<false><<<grid, block, smem, s>>>(g, a, gr);
  }
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_project_backward(const PanelGeom& g, const CamTable& cams, const ProjectArgs& a,
                                    const BlendGrads& gr, const ParamGrads& out, cudaStream_t s) {
  if (a.M == 0) return cudaSuccess;
  k_project_backward<<<(unsigned)((a.M + 127) / 128), 128, 0, s>>>(g, cams, a, gr, out);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace lfd
