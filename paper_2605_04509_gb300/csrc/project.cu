// Projection with cross-view coherent attribute reuse (Sec. 4.2, Eq. 5-6;
// Alg. 1 stage 1). One thread per Gaussian: the 3D covariance is built once
// and the block's SH records are staged in shared memory (coalesced loads,
// widened to FP32; a record per thread at a stride of 49 words, so the lanes
// reading one coefficient hit 32 different banks), then for every cluster k the representative
// view gives the 2D covariance (EWA splatting with the 3DGS Jacobian clamp and
// +0.3 low-pass), its inverse (conic), the depth and the SH colour, and every
// slot view of the cluster gives a 2D mean (Eq. 5). FP32 throughout.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lfd_internal.h"

namespace lfd {
namespace {

// Attribute storage types: FP32, FP16 or BF16, widened to FP32 on load.
__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }

constexpr float kNear = 0.2f;
constexpr float kDilation = 0.3f;

// Real SH basis constants of degree <= 3 (3DGS basis):
// 1/(2 sqrt(pi)), sqrt(3/(4 pi)), sqrt(15/pi)/2, sqrt(5/pi)/4, sqrt(15/pi)/4,
// sqrt(35/(2 pi))/4, sqrt(105/pi)/2, sqrt(21/(2 pi))/4, sqrt(7/pi)/4,
// sqrt(105/pi)/4.
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

__device__ __forceinline__ float3 cam_point(const float* c, float x, float y, float z) {
  return make_float3(c[0] * x + c[1] * y + c[2] * z + c[9], c[3] * x + c[4] * y + c[5] * z + c[10],
                     c[6] * x + c[7] * y + c[8] * z + c[11]);
}

// View-space depth as the bits of the sort key's 32-bit float (Eq. 11):
// ((R20 mx + R21 my) + R22 mz) + t2, each operation rounded to float in this
// order. The depth order and the near-plane test are integer decisions taken
// from this value, so it is evaluated without contraction.
__device__ __forceinline__ float depth_rn(const float* c, float x, float y, float z) {
  return __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(c[6], x), __fmul_rn(c[7], y)), __fmul_rn(c[8], z)),
                   c[11]);
}

constexpr int kProjThreads = 128;
constexpr int kShStride = 49;  // words per staged SH record (48 values, padded)

template <typename A>
__global__ void __launch_bounds__(kProjThreads) k_project(PanelGeom g, CamTable cams, ProjectArgs a) {
  __shared__ float s_sh[kProjThreads * kShStride];
  const int64_t b0 = a.m_begin + (int64_t)blockIdx.x * kProjThreads;  // the block's first Gaussian
  const int64_t i = b0 + threadIdx.x;
  const A* quats = reinterpret_cast<const A*>(a.quats);
  const A* scales = reinterpret_cast<const A*>(a.scales);
  const A* opac = reinterpret_cast<const A*>(a.opac);
  const A* shs = reinterpret_cast<const A*>(a.sh);
  {
    // the block's SH records into shared memory, zeros past the degree
    const int nb = (int)min((int64_t)kProjThreads, a.m_end - b0);
    const int ncoef = (a.sh_degree + 1) * (a.sh_degree + 1);
    const int nv = ncoef * 3;
    constexpr int kPerVec = 16 / (int)sizeof(A);
    if (ncoef == 16 && (reinterpret_cast<uintptr_t>(shs) & 15) == 0) {
      // degree 3: the records are one contiguous run of 48 nb values
      const uint4* src = reinterpret_cast<const uint4*>(shs + (size_t)b0 * 48);
      for (int v = threadIdx.x; v < nb * 48 / kPerVec; v += kProjThreads) {
        const uint4 w = src[v];
        const A* e = reinterpret_cast<const A*>(&w);
#pragma unroll
        for (int q = 0; q < kPerVec; ++q) {
          const int f = v * kPerVec + q;  // value f of the run: record f / 48
          s_sh[(f / 48) * kShStride + f % 48] = to_f32(e[q]);
        }
      }
    } else {
      for (int f = threadIdx.x; f < nb * 48; f += kProjThreads) {
        const int r = f / 48, c = f % 48;
        s_sh[r * kShStride + c] = c < nv ? to_f32(shs[((size_t)b0 + r) * nv + c]) : 0.f;
      }
    }
  }
  __syncthreads();
  if (i >= a.m_end) return;
  const float* sh = s_sh + threadIdx.x * kShStride;  // sh[3 c + u]
  const float mx = a.means[3 * i], my = a.means[3 * i + 1], mz = a.means[3 * i + 2];
  const float4 q4 = make_float4(to_f32(quats[4 * i]), to_f32(quats[4 * i + 1]), to_f32(quats[4 * i + 2]),
                                to_f32(quats[4 * i + 3]));
  const float sx = to_f32(scales[3 * i]), sy = to_f32(scales[3 * i + 1]), sz = to_f32(scales[3 * i + 2]);
  const float o = to_f32(opac[i]);

  // Sigma3D = Rq diag(s^2) Rq^T
  const float qn = rsqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
  const float qw = q4.x * qn, qx = q4.y * qn, qy = q4.z * qn, qz = q4.w * qn;
  const float r00 = 1.f - 2.f * (qy * qy + qz * qz), r01 = 2.f * (qx * qy - qw * qz),
              r02 = 2.f * (qx * qz + qw * qy);
  const float r10 = 2.f * (qx * qy + qw * qz), r11 = 1.f - 2.f * (qx * qx + qz * qz),
              r12 = 2.f * (qy * qz - qw * qx);
  const float r20 = 2.f * (qx * qz - qw * qy), r21 = 2.f * (qy * qz + qw * qx),
              r22 = 1.f - 2.f * (qx * qx + qy * qy);
  const float s0 = sx * sx, s1 = sy * sy, s2 = sz * sz;
  const float S00 = r00 * r00 * s0 + r01 * r01 * s1 + r02 * r02 * s2;
  const float S01 = r00 * r10 * s0 + r01 * r11 * s1 + r02 * r12 * s2;
  const float S02 = r00 * r20 * s0 + r01 * r21 * s1 + r02 * r22 * s2;
  const float S11 = r10 * r10 * s0 + r11 * r11 * s1 + r12 * r12 * s2;
  const float S12 = r10 * r20 * s0 + r11 * r21 * s1 + r12 * r22 * s2;
  const float S22 = r20 * r20 * s0 + r21 * r21 * s1 + r22 * r22 * s2;

  const bool opaque_enough = (double)o >= 1.0 / 255.0;
  const float tau_i = 2.f * logf(255.f * o);
  const float nanf_ = __int_as_float(0x7fc00000);

  for (int k = 0; k < g.K; ++k) {
    const int jr = min(k * g.C + g.C / 2, g.N - 1);
    const float* cr = cams.c[jr];
    float3 p = cam_point(cr, mx, my, mz);
    p.z = depth_rn(cr, mx, my, mz);
    const size_t ok = (size_t)k * a.M + i;
    float4 co = make_float4(0.f, 0.f, 0.f, o);
    float4 ct = make_float4(0.f, 0.f, 0.f, -1.f);
    if (p.z > kNear && opaque_enough) {
      const float fx = cr[12], fy = cr[13];
      const float limx = 1.3f * (0.5f * (float)g.W / fx);
      const float limy = 1.3f * (0.5f * (float)g.H / fy);
      const float iz = 1.f / p.z;
      const float txz = fminf(fmaxf(p.x * iz, -limx), limx);
      const float tyz = fminf(fmaxf(p.y * iz, -limy), limy);
      const float j00 = fx * iz, j02 = -fx * txz * iz;
      const float j11 = fy * iz, j12 = -fy * tyz * iz;
      // T = J R_cam (2 x 3)
      const float t00 = j00 * cr[0] + j02 * cr[6];
      const float t01 = j00 * cr[1] + j02 * cr[7];
      const float t02 = j00 * cr[2] + j02 * cr[8];
      const float t10 = j11 * cr[3] + j12 * cr[6];
      const float t11 = j11 * cr[4] + j12 * cr[7];
      const float t12 = j11 * cr[5] + j12 * cr[8];
      // U = T Sigma3D
      const float u00 = t00 * S00 + t01 * S01 + t02 * S02;
      const float u01 = t00 * S01 + t01 * S11 + t02 * S12;
      const float u02 = t00 * S02 + t01 * S12 + t02 * S22;
      const float u10 = t10 * S00 + t11 * S01 + t12 * S02;
      const float u11 = t10 * S01 + t11 * S11 + t12 * S12;
      const float u12 = t10 * S02 + t11 * S12 + t12 * S22;
      const float cxx = u00 * t00 + u01 * t01 + u02 * t02 + kDilation;
      const float cxy = u00 * t10 + u01 * t11 + u02 * t12;
      const float cyy = u10 * t10 + u11 * t11 + u12 * t12 + kDilation;
      const float det = cxx * cyy - cxy * cxy;
      if (det > 0.f) {
        const float id = 1.f / det;
        co = make_float4(cyy * id, -cxy * id, cxx * id, o);
        // colour at the representative camera centre c = -R^T t
        const float px = -(cr[0] * cr[9] + cr[3] * cr[10] + cr[6] * cr[11]);
        const float py = -(cr[1] * cr[9] + cr[4] * cr[10] + cr[7] * cr[11]);
        const float pz = -(cr[2] * cr[9] + cr[5] * cr[10] + cr[8] * cr[11]);
        float dx = mx - px, dy = my - py, dz = mz - pz;
        const float dn = rsqrtf(dx * dx + dy * dy + dz * dz);
        dx *= dn;
        dy *= dn;
        dz *= dn;
        const float xx = dx * dx, yy = dy * dy, zz = dz * dz;
        float b[16];
        b[0] = kC0;
        b[1] = -kC1 * dy;
        b[2] = kC1 * dz;
        b[3] = -kC1 * dx;
        b[4] = kC2a * dx * dy;
        b[5] = -kC2a * dy * dz;
        b[6] = kC2b * (2.f * zz - xx - yy);
        b[7] = -kC2a * dx * dz;
        b[8] = kC2c * (xx - yy);
        b[9] = -kC3a * dy * (3.f * xx - yy);
        b[10] = kC3b * dx * dy * dz;
        b[11] = -kC3c * dy * (4.f * zz - xx - yy);
        b[12] = kC3d * dz * (2.f * zz - 3.f * xx - 3.f * yy);
        b[13] = -kC3c * dx * (4.f * zz - xx - yy);
        b[14] = kC3e * dz * (xx - yy);
        b[15] = -kC3a * dx * (xx - 3.f * yy);
        float rgb[3];
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          float acc = 0.f;
#pragma unroll
          for (int c = 0; c < 16; ++c) acc += b[c] * sh[3 * c + u];
          rgb[u] = fmaxf(acc + 0.5f, 0.f);
        }
        ct = make_float4(rgb[0], rgb[1], rgb[2], tau_i);
      }
    }
    reinterpret_cast<float4*>(a.conic_opacity)[ok] = co;
    reinterpret_cast<float4*>(a.color_tau)[ok] = ct;
    a.depth[ok] = p.z;
    // Eq. 5: per-view 2D means of every slot of the cluster
    float2* mo = reinterpret_cast<float2*>(a.means2d) + ok * g.C;
    auto mean_of = [&](int l) -> float2 {
      const int j = min(k * g.C + l, g.N - 1);
      const float* cj = cams.c[j];
      const float3 pj = cam_point(cj, mx, my, mz);
      float2 m2 = make_float2(nanf_, nanf_);
      if (depth_rn(cj, mx, my, mz) > kNear) {
        const float iz = 1.f / pj.z;
        m2 = make_float2(cj[12] * pj.x * iz + cj[14], cj[13] * pj.y * iz + cj[15]);
      }
      return m2;
    };
    if ((g.C & 1) == 0 && (reinterpret_cast<uintptr_t>(mo) & 15) == 0) {
      // two views per 16-byte store
      for (int l = 0; l < g.C; l += 2) {
        const float2 m0 = mean_of(l), m1 = mean_of(l + 1);
        reinterpret_cast<float4*>(mo)[l >> 1] = make_float4(m0.x, m0.y, m1.x, m1.y);
      }
    } else {
      for (int l = 0; l < g.C; ++l) mo[l] = mean_of(l);
    }
  }
}

}  // namespace

cudaError_t launch_project(const PanelGeom& g, const CamTable& cams, const ProjectArgs& args,
                           cudaStream_t s) {
  ProjectArgs a = args;
  if (a.m_end < 0 || a.m_end > a.M) a.m_end = a.M;
  if (a.m_begin < 0) a.m_begin = 0;
  if (a.m_end <= a.m_begin) return cudaSuccess;
  const int threads = kProjThreads;
  const int64_t blocks = (a.m_end - a.m_begin + threads - 1) / threads;
  if (a.attr_dtype == LFD_DTYPE_F16)
    k_project<__half><<<(unsigned)blocks, threads, 0, s>>>(g, cams, a);
  else if (a.attr_dtype == LFD_DTYPE_BF16)
    k_project<__nv_bfloat16><<<(unsigned)blocks, threads, 0, s>>>(g, cams, a);
  else
    k_project<float><<<(unsigned)blocks, threads, 0, s>>>(g, cams, a);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace lfd
