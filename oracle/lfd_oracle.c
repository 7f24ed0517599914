/*
 * Plain CPU oracle for subpixel-level 3DGS rasterisation of an interlaced
 * light-field image (CoherentRaster, arXiv 2605.04509).
 *
 * TEST INFRASTRUCTURE ONLY: called from the tests, the smoke check and the
 * benchmark's CPU baseline; never from the product path. It shares no code
 * with the CUDA library. Build: gcc -O2 -std=c11 -fopenmp -fPIC -shared
 * -ffp-contract=off (no contraction: every FP operation is rounded on its own,
 * which the FP32 mirror needs for bit-exact tile bins).
 *
 * Parity status per function (what pins it lives in tests/test_oracle_*.py):
 *   orc_view_index      pinned: exact rational evaluation of Eq. 1-3.
 *   orc_remap           pinned: permutation + Eq. 8 monotonicity + stability.
 *   orc_clusters        pinned: Appendix B.1 tables written out by hand.
 *   orc_project         pinned: closed forms (on-axis isotropic Gaussian),
 *                       finite-difference Jacobian, rotation matrices from an
 *                       independent library, real SH from Legendre functions.
 *   orc_render          pinned: single- and two-Gaussian closed forms, the
 *                       termination rule, a vectorised textbook 3DGS renderer
 *                       (one view), full-frame + interlace (C = 1), mode 0 vs 1.
 *   orc_blend_lists     pinned against orc_render on the same lists.
 *   orc_render_fullframe  pinned against the vectorised textbook renderer.
 *   orc_mirror_*        pinned: brute-force pixel scans of the region
 *                       {q <= tau} (superset and tightness), Eq. 11 decoding,
 *                       sortedness and range invariants.
 *   Attribute reuse across a cluster (Eq. 6) is an approximation with no
 *   closed form: its image is pinned only through the C = 1 identity; the
 *   quality loss for C > 1 is "parity unpinned" against the paper's numbers.
 */
#include "lfd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NEAR_PLANE 0.2
#define DILATION 0.3
/* skip threshold of Eq. 10's alpha (3DGS: 1/255); settable for sensitivity
 * analysis of the definition, see orc_set_alpha_min */
static double g_alpha_min = 1.0 / 255.0;
#define ALPHA_MIN g_alpha_min
#define ALPHA_MAX 0.99
#define T_MIN 1e-4

double orc_set_alpha_min(double v) {
  const double old = g_alpha_min;
  if (v > 0.0) g_alpha_min = v;
  return old;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

static int num_clusters(int N, int C) { return (N + C - 1) / C; }

/* ------------------------------------------------------------------ */
/* Sec. 3.1, Eq. 1-3: view index matrix.                                */
/* d = 3x + u + 3y tan(alpha) - K_off; x_off = d mod L_x (floored);    */
/* j = floor(N x_off / L_x), clamped to [0, N-1] against rounding.     */
/* ------------------------------------------------------------------ */
int orc_view_index(int W, int H, int N, double tan_slant, double pitch,
                   double k_offset, uint8_t *V) {
  if (W <= 0 || H <= 0 || N <= 0 || N > 255 || !(pitch > 0.0)) return -1;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < H; ++y) {
    for (int x = 0; x < W; ++x) {
      for (int u = 0; u < 3; ++u) {
        double col = 3.0 * (double)x;
        col = col + (double)u;
        double row = 3.0 * (double)y;
        row = row * tan_slant;
        double d = col + row;
        d = d - k_offset;
        double q = floor(d / pitch);
        double xoff = d - pitch * q;
        double r = ((double)N * xoff) / pitch;
        int j = (int)floor(r);
        if (j < 0) j = 0;
        if (j > N - 1) j = N - 1;
        V[((size_t)y * W + x) * 3 + u] = (uint8_t)j;
      }
    }
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Sec. 4.3, Eq. 8: for each tile, the in-panel subpixels in row-major  */
/* order, stably sorted by view index. seg[t][k] is the first position */
/* whose view belongs to cluster >= k.                                  */
/* ------------------------------------------------------------------ */
int orc_remap(int W, int H, int N, const uint8_t *V, int TW, int TH, int C,
              uint16_t *psi, int32_t *n_sub, int32_t *seg) {
  if (TW <= 0 || TH <= 0 || C <= 0 || TW * TH * 3 > 65536) return -1;
  const int TX = (W + TW - 1) / TW, TY = (H + TH - 1) / TH;
  const int K = num_clusters(N, C);
  const int cap = TW * TH * 3;
#pragma omp parallel for schedule(dynamic, 16)
  for (int t = 0; t < TX * TY; ++t) {
    const int tx = t % TX, ty = t / TX;
    int hist[256];
    int start[257];
    memset(hist, 0, sizeof(hist));
    for (int yl = 0; yl < TH; ++yl) {
      const int y = ty * TH + yl;
      if (y >= H) break;
      for (int xl = 0; xl < TW; ++xl) {
        const int x = tx * TW + xl;
        if (x >= W) break;
        for (int u = 0; u < 3; ++u) hist[V[((size_t)y * W + x) * 3 + u]]++;
      }
    }
    start[0] = 0;
    for (int j = 0; j < 256; ++j) start[j + 1] = start[j] + hist[j];
    n_sub[t] = start[256];
    for (int k = 0; k <= K; ++k) {
      int jv = k * C;
      if (jv > 256) jv = 256;
      seg[(size_t)t * (K + 1) + k] = start[jv];
    }
    seg[(size_t)t * (K + 1) + K] = start[256];
    int fill[256];
    for (int j = 0; j < 256; ++j) fill[j] = start[j];
    uint16_t *dst = psi + (size_t)t * cap;
    for (int yl = 0; yl < TH; ++yl) {
      const int y = ty * TH + yl;
      if (y >= H) break;
      for (int xl = 0; xl < TW; ++xl) {
        const int x = tx * TW + xl;
        if (x >= W) break;
        for (int u = 0; u < 3; ++u) {
          const int j = V[((size_t)y * W + x) * 3 + u];
          dst[fill[j]++] = (uint16_t)((yl * TW + xl) * 3 + u);
        }
      }
    }
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Appendix B.1: contiguous clusters of C views along the trajectory;   */
/* the last one is padded by repeating view N-1; the representative is */
/* the camera at local index floor(C/2).                                */
/* ------------------------------------------------------------------ */
int orc_clusters(int N, int C, int32_t *slot_view, int32_t *rep) {
  if (N <= 0 || C <= 0) return -1;
  const int K = num_clusters(N, C);
  for (int k = 0; k < K; ++k) {
    for (int l = 0; l < C; ++l) {
      int j = k * C + l;
      slot_view[k * C + l] = j < N ? j : N - 1;
    }
    rep[k] = slot_view[k * C + C / 2];
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Sec. 3.3, Eq. 4-6: projection in FP64.                               */
/* ------------------------------------------------------------------ */
typedef struct {
  double R[9], t[3], fx, fy, cx, cy;
} cam64;

static void load_cam(const float *c, cam64 *o) {
  for (int a = 0; a < 9; ++a) o->R[a] = c[a];
  for (int a = 0; a < 3; ++a) o->t[a] = c[9 + a];
  o->fx = c[12];
  o->fy = c[13];
  o->cx = c[14];
  o->cy = c[15];
}

/* View-space depth in FP32, each operation rounded in this fixed order:
 * ((R20 mx + R21 my) + R22 mz) + t2. Eq. 11 stores the depth of the sort
 * key as the bits of a 32-bit float, so the depth order (and with it the
 * near-plane test) is decided in FP32 by this one sequence; everything else
 * in the oracle stays FP64. */
static float depth_f32(const float *cam, const float *m) {
  const float a0 = cam[6] * m[0];
  const float a1 = cam[7] * m[1];
  const float a2 = cam[8] * m[2];
  float d = a0 + a1;
  d = d + a2;
  d = d + cam[11];
  return d;
}

static void to_camera(const cam64 *c, const double m[3], double p[3]) {
  for (int r = 0; r < 3; ++r)
    p[r] = c->R[3 * r + 0] * m[0] + c->R[3 * r + 1] * m[1] +
           c->R[3 * r + 2] * m[2] + c->t[r];
}

/* Real spherical harmonics up to degree 3 in the basis and sign convention
 * of 3DGS: for m != 0 the functions are sqrt(2) Re / Im of the complex
 * Y_l^m with the Condon-Shortley phase, ordered m = -l..l. The constants are
 * written from their closed forms. */
static void sh_basis(double x, double y, double z, double b[16]) {
  const double pi = 3.14159265358979323846;
  const double c0 = 0.5 * sqrt(1.0 / pi);
  const double c1 = sqrt(3.0 / (4.0 * pi));
  const double c2a = 0.5 * sqrt(15.0 / pi);
  const double c2b = 0.25 * sqrt(5.0 / pi);
  const double c2c = 0.25 * sqrt(15.0 / pi);
  const double c3a = 0.25 * sqrt(35.0 / (2.0 * pi));
  const double c3b = 0.5 * sqrt(105.0 / pi);
  const double c3c = 0.25 * sqrt(21.0 / (2.0 * pi));
  const double c3d = 0.25 * sqrt(7.0 / pi);
  const double c3e = 0.25 * sqrt(105.0 / pi);
  const double xx = x * x, yy = y * y, zz = z * z;
  b[0] = c0;
  b[1] = -c1 * y;
  b[2] = c1 * z;
  b[3] = -c1 * x;
  b[4] = c2a * x * y;
  b[5] = -c2a * y * z;
  b[6] = c2b * (2.0 * zz - xx - yy);
  b[7] = -c2a * x * z;
  b[8] = c2c * (xx - yy);
  b[9] = -c3a * y * (3.0 * xx - yy);
  b[10] = c3b * x * y * z;
  b[11] = -c3c * y * (4.0 * zz - xx - yy);
  b[12] = c3d * z * (2.0 * zz - 3.0 * xx - 3.0 * yy);
  b[13] = -c3c * x * (4.0 * zz - xx - yy);
  b[14] = c3e * z * (xx - yy);
  b[15] = -c3a * x * (xx - 3.0 * yy);
}

int orc_project(int64_t M, const float *means, const float *scales,
                const float *quats, const float *opac, const float *sh,
                int sh_degree, int N, const float *cams, int W, int H, int C,
                double *mean2d, uint8_t *vvalid, double *conic, double *depth,
                double *color, double *tau, uint8_t *valid) {
  if (M < 0 || N <= 0 || C <= 0 || sh_degree < 0 || sh_degree > 3) return -1;
  const int K = num_clusters(N, C);
  const int ncoef = (sh_degree + 1) * (sh_degree + 1);
  cam64 *cv = (cam64 *)malloc(sizeof(cam64) * (size_t)N);
  if (!cv) return -2;
  for (int j = 0; j < N; ++j) load_cam(cams + 16 * j, &cv[j]);

  /* Eq. 5: 2D mean of every Gaussian in every view. */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < M; ++i) {
    const double m[3] = {means[3 * i], means[3 * i + 1], means[3 * i + 2]};
    for (int j = 0; j < N; ++j) {
      double p[3];
      to_camera(&cv[j], m, p);
      const size_t o = (size_t)j * M + i;
      if (depth_f32(cams + 16 * j, means + 3 * i) > (float)NEAR_PLANE) {
        vvalid[o] = 1;
        mean2d[2 * o] = cv[j].fx * p[0] / p[2] + cv[j].cx;
        mean2d[2 * o + 1] = cv[j].fy * p[1] / p[2] + cv[j].cy;
      } else {
        vvalid[o] = 0;
        mean2d[2 * o] = 0.0;
        mean2d[2 * o + 1] = 0.0;
      }
    }
  }

  /* Eq. 6: covariance, depth and colour at each cluster representative. */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < M; ++i) {
    const double m[3] = {means[3 * i], means[3 * i + 1], means[3 * i + 2]};
    double qw = quats[4 * i], qx = quats[4 * i + 1], qy = quats[4 * i + 2],
           qz = quats[4 * i + 3];
    const double qn = sqrt(qw * qw + qx * qx + qy * qy + qz * qz);
    qw /= qn;
    qx /= qn;
    qy /= qn;
    qz /= qn;
    const double Rq[9] = {1.0 - 2.0 * (qy * qy + qz * qz), 2.0 * (qx * qy - qw * qz),
                          2.0 * (qx * qz + qw * qy),       2.0 * (qx * qy + qw * qz),
                          1.0 - 2.0 * (qx * qx + qz * qz), 2.0 * (qy * qz - qw * qx),
                          2.0 * (qx * qz - qw * qy),       2.0 * (qy * qz + qw * qx),
                          1.0 - 2.0 * (qx * qx + qy * qy)};
    const double s[3] = {scales[3 * i], scales[3 * i + 1], scales[3 * i + 2]};
    double S3[9]; /* Sigma = Rq diag(s^2) Rq^T */
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        double acc = 0.0;
        for (int a = 0; a < 3; ++a) acc += Rq[3 * r + a] * s[a] * s[a] * Rq[3 * c + a];
        S3[3 * r + c] = acc;
      }
    const double o = opac[i];
    for (int k = 0; k < K; ++k) {
      int jr = k * C + C / 2;
      if (jr > N - 1) jr = N - 1;
      const cam64 *cr = &cv[jr];
      double p[3];
      to_camera(cr, m, p);
      const size_t ok = (size_t)k * M + i;
      valid[ok] = 0;
      conic[3 * ok] = conic[3 * ok + 1] = conic[3 * ok + 2] = 0.0;
      color[3 * ok] = color[3 * ok + 1] = color[3 * ok + 2] = 0.0;
      const float zkey = depth_f32(cams + 16 * jr, means + 3 * i);
      depth[ok] = (double)zkey;
      tau[ok] = -1.0;
      if (!(zkey > (float)NEAR_PLANE)) continue;
      /* Jacobian of the pinhole projection, with the 3DGS clamp of x/z and
       * y/z to 1.3 times the half field of view. */
      const double limx = 1.3 * (0.5 * (double)W / cr->fx);
      const double limy = 1.3 * (0.5 * (double)H / cr->fy);
      double txz = p[0] / p[2], tyz = p[1] / p[2];
      txz = txz < -limx ? -limx : (txz > limx ? limx : txz);
      tyz = tyz < -limy ? -limy : (tyz > limy ? limy : tyz);
      const double J[6] = {cr->fx / p[2], 0.0, -cr->fx * txz / p[2],
                           0.0, cr->fy / p[2], -cr->fy * tyz / p[2]};
      double T[6]; /* J R_cam */
      for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c)
          T[3 * r + c] = J[3 * r] * cr->R[c] + J[3 * r + 1] * cr->R[3 + c] +
                         J[3 * r + 2] * cr->R[6 + c];
      double S2[4];
      for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
          double acc = 0.0;
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) acc += T[3 * r + a] * S3[3 * a + b] * T[3 * c + b];
          S2[2 * r + c] = acc;
        }
      S2[0] += DILATION;
      S2[3] += DILATION;
      const double det = S2[0] * S2[3] - S2[1] * S2[2];
      if (!(det > 0.0)) continue;
      if (!(o >= ALPHA_MIN)) continue;
      conic[3 * ok] = S2[3] / det;
      conic[3 * ok + 1] = -S2[1] / det;
      conic[3 * ok + 2] = S2[0] / det;
      tau[ok] = 2.0 * log(255.0 * o);
      /* view-dependent colour at the representative camera centre */
      const double cpos[3] = {
          -(cr->R[0] * cr->t[0] + cr->R[3] * cr->t[1] + cr->R[6] * cr->t[2]),
          -(cr->R[1] * cr->t[0] + cr->R[4] * cr->t[1] + cr->R[7] * cr->t[2]),
          -(cr->R[2] * cr->t[0] + cr->R[5] * cr->t[1] + cr->R[8] * cr->t[2])};
      double dx = m[0] - cpos[0], dy = m[1] - cpos[1], dz = m[2] - cpos[2];
      const double dn = sqrt(dx * dx + dy * dy + dz * dz);
      dx /= dn;
      dy /= dn;
      dz /= dn;
      double bas[16];
      sh_basis(dx, dy, dz, bas);
      for (int u = 0; u < 3; ++u) {
        double acc = 0.0;
        for (int cidx = 0; cidx < ncoef; ++cidx)
          acc += bas[cidx] * sh[((size_t)i * ncoef + cidx) * 3 + u];
        acc += 0.5;
        color[3 * ok + u] = acc > 0.0 ? acc : 0.0;
      }
      valid[ok] = 1;
    }
  }
  free(cv);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Eq. 9-10: front-to-back blend of one subpixel along a list, with the */
/* 3DGS rules: alpha = min(0.99, o exp(-q/2)); skip alpha < 1/255; stop */
/* (without adding) once the transmittance would fall below 1e-4.       */
/* ------------------------------------------------------------------ */
typedef struct {
  int64_t M;
  const double *mean2d;
  const uint8_t *vvalid;
  const double *conic;
  const double *color;
  const double *opac;
} blend_in;

static double blend_walk(const blend_in *b, const uint32_t *idx, int64_t n,
                         double px, double py, int u, int j, int k, double bg,
                         int64_t *cnt) {
  double T = 1.0, acc = 0.0;
  int64_t visited = 0;
  for (int64_t e = 0; e < n; ++e) {
    const uint32_t i = idx[e];
    ++visited;
    const size_t ov = (size_t)j * b->M + i;
    if (!b->vvalid[ov]) continue;
    const size_t ok = (size_t)k * b->M + i;
    const double dx = px - b->mean2d[2 * ov];
    const double dy = py - b->mean2d[2 * ov + 1];
    const double ca = b->conic[3 * ok], cb = b->conic[3 * ok + 1], cc = b->conic[3 * ok + 2];
    const double q = ca * dx * dx + 2.0 * cb * dx * dy + cc * dy * dy;
    const double power = -0.5 * q;
    if (power > 0.0) continue;
    const double v = b->opac[i] * exp(power);
    if (v < ALPHA_MIN) continue;
    const double alpha = v < ALPHA_MAX ? v : ALPHA_MAX;
    const double Tn = T * (1.0 - alpha);
    if (Tn < T_MIN) break;
    acc += b->color[3 * ok + u] * alpha * T;
    T = Tn;
  }
  if (cnt) *cnt += visited;
  return acc + T * bg;
}

/* (depth, id) order of the valid Gaussians of one cluster */
typedef struct {
  double d;
  uint32_t i;
} dkey;

static int cmp_dkey(const void *a, const void *b) {
  const dkey *x = (const dkey *)a, *y = (const dkey *)b;
  if (x->d < y->d) return -1;
  if (x->d > y->d) return 1;
  return (x->i > y->i) - (x->i < y->i);
}

static uint32_t *depth_order(int64_t M, const double *depth, const uint8_t *valid,
                             int64_t *count) {
  dkey *tmp = (dkey *)malloc(sizeof(dkey) * (size_t)(M > 0 ? M : 1));
  int64_t n = 0;
  for (int64_t i = 0; i < M; ++i)
    if (valid[i]) {
      tmp[n].d = depth[i];
      tmp[n].i = (uint32_t)i;
      ++n;
    }
  qsort(tmp, (size_t)n, sizeof(dkey), cmp_dkey);
  uint32_t *out = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t e = 0; e < n; ++e) out[e] = tmp[e].i;
  free(tmp);
  *count = n;
  return out;
}

int orc_render(int W, int H, int N, int C, const uint8_t *V, int TW, int TH,
               int64_t M, const double *mean2d, const uint8_t *vvalid,
               const double *conic, const double *depth, const double *color,
               const uint8_t *valid, const double *opac, int x0, int y0,
               int x1, int y1, int mode, const double *bg, double *out,
               int64_t *n_eval) {
  if (x0 < 0 || y0 < 0 || x1 > W || y1 > H || x0 > x1 || y0 > y1 || C <= 0)
    return -1;
  const int K = num_clusters(N, C);
  const int cw = x1 - x0;
  blend_in bi = {M, mean2d, vvalid, conic, color, opac};
  uint32_t **ord = (uint32_t **)calloc((size_t)K, sizeof(uint32_t *));
  int64_t *nord = (int64_t *)calloc((size_t)K, sizeof(int64_t));
  for (int k = 0; k < K; ++k)
    ord[k] = depth_order(M, depth + (size_t)k * M, valid + (size_t)k * M, &nord[k]);
  int64_t total = 0;

  if (mode == 0) {
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total)
    for (int y = y0; y < y1; ++y)
      for (int x = x0; x < x1; ++x)
        for (int u = 0; u < 3; ++u) {
          const int j = V[((size_t)y * W + x) * 3 + u];
          const int k = j / C;
          out[((size_t)(y - y0) * cw + (x - x0)) * 3 + u] =
              blend_walk(&bi, ord[k], nord[k], x + 0.5, y + 0.5, u, j, k, bg[u], &total);
        }
  } else {
    /* Binned: per (tile, cluster) lists from a conservative bounding box of
     * the region {q <= 2 ln(255 o)} (where alpha >= 1/255), widened by one
     * pixel, united over the cluster's views. Lists keep the depth order. */
    if (TW <= 0 || TH <= 0) return -1;
    const int tx0 = x0 / TW, ty0 = y0 / TH;
    const int tx1 = x1 > x0 ? (x1 - 1) / TW : tx0 - 1;
    const int ty1 = y1 > y0 ? (y1 - 1) / TH : ty0 - 1;
    const int ntx = tx1 - tx0 + 1, nty = ty1 - ty0 + 1;
    const int nt = ntx > 0 && nty > 0 ? ntx * nty : 0;
    int64_t *cnt = (int64_t *)calloc((size_t)nt * K + 1, sizeof(int64_t));
    int64_t *off = (int64_t *)calloc((size_t)nt * K + 1, sizeof(int64_t));
    for (int pass = 0; pass < 2 && nt > 0; ++pass) {
      uint32_t *lists = NULL;
      if (pass == 1) {
        int64_t s = 0;
        for (int64_t a = 0; a < (int64_t)nt * K; ++a) {
          off[a] = s;
          s += cnt[a];
          cnt[a] = 0;
        }
        lists = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(s > 0 ? s : 1));
      }
      for (int k = 0; k < K; ++k) {
        for (int64_t e = 0; e < nord[k]; ++e) {
          const uint32_t i = ord[k][e];
          const size_t ok = (size_t)k * M + i;
          const double ca = conic[3 * ok], cb = conic[3 * ok + 1], cc = conic[3 * ok + 2];
          const double det = ca * cc - cb * cb;
          if (!(det > 0.0) || !(opac[i] >= ALPHA_MIN)) continue;
          const double tau = 2.0 * log(255.0 * opac[i]);
          const double hx = sqrt(tau * cc / det) + 1.0;
          const double hy = sqrt(tau * ca / det) + 1.0;
          int rx0 = 1 << 30, rx1 = -1, ry0 = 1 << 30, ry1 = -1;
          for (int l = 0; l < C; ++l) {
            int j = k * C + l;
            if (j > N - 1) j = N - 1;
            const size_t ov = (size_t)j * M + i;
            if (!vvalid[ov]) continue;
            const double mx = mean2d[2 * ov], my = mean2d[2 * ov + 1];
            /* pixel columns whose centre lies within [mx-hx, mx+hx] */
            double fa = ceil(mx - hx - 0.5), fb = floor(mx + hx - 0.5);
            double ga = ceil(my - hy - 0.5), gb = floor(my + hy - 0.5);
            if (fa < x0) fa = x0;
            if (fb > x1 - 1) fb = x1 - 1;
            if (ga < y0) ga = y0;
            if (gb > y1 - 1) gb = y1 - 1;
            if (fa > fb || ga > gb) continue;
            const int a0 = (int)fa / TW, a1 = (int)fb / TW;
            const int b0 = (int)ga / TH, b1 = (int)gb / TH;
            if (a0 < rx0) rx0 = a0;
            if (a1 > rx1) rx1 = a1;
            if (b0 < ry0) ry0 = b0;
            if (b1 > ry1) ry1 = b1;
          }
          for (int ty = ry0; ty <= ry1; ++ty)
            for (int tx = rx0; tx <= rx1; ++tx) {
              const size_t slot = ((size_t)(ty - ty0) * ntx + (tx - tx0)) * K + k;
              if (pass == 1) lists[off[slot] + cnt[slot]] = i;
              cnt[slot]++;
            }
        }
      }
      if (pass == 1) {
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total)
        for (int y = y0; y < y1; ++y)
          for (int x = x0; x < x1; ++x)
            for (int u = 0; u < 3; ++u) {
              const int j = V[((size_t)y * W + x) * 3 + u];
              const int k = j / C;
              const size_t slot = ((size_t)(y / TH - ty0) * ntx + (x / TW - tx0)) * K + k;
              out[((size_t)(y - y0) * cw + (x - x0)) * 3 + u] = blend_walk(
                  &bi, lists + off[slot], cnt[slot], x + 0.5, y + 0.5, u, j, k, bg[u], &total);
            }
        free(lists);
      }
    }
    free(cnt);
    free(off);
  }
  for (int k = 0; k < K; ++k) free(ord[k]);
  free(ord);
  free(nord);
  if (n_eval) *n_eval = total;
  return 0;
}

int orc_blend_lists(int W, int H, int N, int C, const uint8_t *V, int TW,
                    int TH, int64_t M, const double *mean2d,
                    const uint8_t *vvalid, const double *conic,
                    const double *color, const double *opac,
                    const uint32_t *ranges, const uint32_t *list, int x0,
                    int y0, int x1, int y1, const double *bg, double *out,
                    int64_t *n_eval) {
  if (x0 < 0 || y0 < 0 || x1 > W || y1 > H || x0 > x1 || y0 > y1 || C <= 0)
    return -1;
  const int K = num_clusters(N, C);
  const int TX = (W + TW - 1) / TW;
  const int cw = x1 - x0;
  blend_in bi = {M, mean2d, vvalid, conic, color, opac};
  int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total)
  for (int y = y0; y < y1; ++y)
    for (int x = x0; x < x1; ++x)
      for (int u = 0; u < 3; ++u) {
        const int j = V[((size_t)y * W + x) * 3 + u];
        const int k = j / C;
        const size_t t = (size_t)(y / TH) * TX + (x / TW);
        const uint32_t s = ranges[(t * K + k) * 2], e = ranges[(t * K + k) * 2 + 1];
        out[((size_t)(y - y0) * cw + (x - x0)) * 3 + u] =
            blend_walk(&bi, list + s, (int64_t)e - s, x + 0.5, y + 0.5, u, j, k, bg[u], &total);
      }
  if (n_eval) *n_eval = total;
  return 0;
}

/* ------------------------------------------------------------------ */
/* Full-frame baseline: render every view as an ordinary 3DGS image,   */
/* one pixel at a time with all three channels, then pick each         */
/* subpixel from the image of its view.                                */
/* ------------------------------------------------------------------ */
int orc_render_fullframe(int W, int H, int N, const uint8_t *V, int64_t M,
                         const double *mean2d, const uint8_t *vvalid,
                         const double *conic, const double *depth,
                         const double *color, const uint8_t *valid,
                         const double *opac, int x0, int y0, int x1, int y1,
                         const double *bg, double *out) {
  if (x0 < 0 || y0 < 0 || x1 > W || y1 > H || x0 > x1 || y0 > y1) return -1;
  const int cw = x1 - x0, ch = y1 - y0;
  const size_t npx = (size_t)cw * ch;
  double *img = (double *)malloc(sizeof(double) * (npx * 3 * (size_t)N + 1));
  for (int j = 0; j < N; ++j) {
    int64_t n;
    uint32_t *ord = depth_order(M, depth + (size_t)j * M, valid + (size_t)j * M, &n);
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = y0; y < y1; ++y)
      for (int x = x0; x < x1; ++x) {
        double T = 1.0, acc[3] = {0.0, 0.0, 0.0};
        for (int64_t e = 0; e < n; ++e) {
          const uint32_t i = ord[e];
          const size_t o = (size_t)j * M + i;
          if (!vvalid[o]) continue;
          const double dx = (x + 0.5) - mean2d[2 * o];
          const double dy = (y + 0.5) - mean2d[2 * o + 1];
          const double q = conic[3 * o] * dx * dx + 2.0 * conic[3 * o + 1] * dx * dy +
                           conic[3 * o + 2] * dy * dy;
          const double power = -0.5 * q;
          if (power > 0.0) continue;
          const double v = opac[i] * exp(power);
          if (v < ALPHA_MIN) continue;
          const double alpha = v < ALPHA_MAX ? v : ALPHA_MAX;
          const double Tn = T * (1.0 - alpha);
          if (Tn < T_MIN) break;
          for (int u = 0; u < 3; ++u) acc[u] += color[3 * o + u] * alpha * T;
          T = Tn;
        }
        double *px = img + ((size_t)j * npx + (size_t)(y - y0) * cw + (x - x0)) * 3;
        for (int u = 0; u < 3; ++u) px[u] = acc[u] + T * bg[u];
      }
    free(ord);
  }
  for (int y = y0; y < y1; ++y)
    for (int x = x0; x < x1; ++x)
      for (int u = 0; u < 3; ++u) {
        const int j = V[((size_t)y * W + x) * 3 + u];
        const size_t p = (size_t)(y - y0) * cw + (x - x0);
        out[p * 3 + u] = img[((size_t)j * npx + p) * 3 + u];
      }
  free(img);
  (void)H;
  return 0;
}

/* ------------------------------------------------------------------ */
/* FP32 mirror of the tile-bin rule (Alg. 2, GenerateKeys). The region  */
/* of Gaussian i in view j is {p : q(p - mu_ij) <= tau_ik}, the set of  */
/* pixel centres where alpha >= 1/255 (Eq. 10). For every tile row the  */
/* exact x-extent of the ellipse over that row's band of pixel-centre   */
/* heights is taken (the extreme lies at the clamp of the ellipse's     */
/* rightmost / leftmost point into the band); a tile is hit when a      */
/* pixel-centre column inside that extent falls in it. All arithmetic   */
/* is float32, each operation correctly rounded, in the order written.  */
/* ------------------------------------------------------------------ */
typedef struct {
  float a, b, c, tau, det, hx, hy, ys, ia;
} binq;

static int bin_prep(float a, float b, float c, float tau, binq *o) {
  if (!isfinite(a) || !isfinite(b) || !isfinite(c) || !isfinite(tau)) return 0;
  if (!(tau >= 0.0f) || !(a > 0.0f) || !(c > 0.0f)) return 0;
  const float ac = a * c;
  const float bb = b * b;
  const float det = ac - bb;
  if (!(det > 0.0f)) return 0;
  o->a = a;
  o->b = b;
  o->c = c;
  o->tau = tau;
  o->det = det;
  const float ta = tau * a;
  const float tc = tau * c;
  o->hy = sqrtf(ta / det);
  o->hx = sqrtf(tc / det);
  const float dc = det * c;
  const float r = sqrtf(tau / dc);
  o->ys = b * r;
  o->ia = 1.0f / a;
  return 1;
}

typedef struct {
  int valid;
  float mx, my;
  int y0, y1;   /* pixel rows, inclusive */
  float bx0, bx1; /* pixel columns of the bounding box, inclusive */
} binv;

static void bin_view(const binq *g, float mx, float my, int W, int H, binv *v) {
  v->valid = 0;
  if (!isfinite(mx) || !isfinite(my)) return;
  const float ylo = my - g->hy;
  const float yhi = my + g->hy;
  float fy0 = ceilf(ylo - 0.5f);
  float fy1 = floorf(yhi - 0.5f);
  fy0 = fmaxf(fy0, 0.0f);
  fy1 = fminf(fy1, (float)(H - 1));
  const float xlo = mx - g->hx;
  const float xhi = mx + g->hx;
  float fx0 = ceilf(xlo - 0.5f);
  float fx1 = floorf(xhi - 0.5f);
  fx0 = fmaxf(fx0, 0.0f);
  fx1 = fminf(fx1, (float)(W - 1));
  if (!(fy0 <= fy1) || !(fx0 <= fx1)) return;
  v->valid = 1;
  v->mx = mx;
  v->my = my;
  v->y0 = (int)fy0;
  v->y1 = (int)fy1;
  v->bx0 = fx0;
  v->bx1 = fx1;
}

/* tile-column interval of view v in tile row ty; returns 0 if empty */
static int bin_row(const binq *g, const binv *v, int ty, int TW, int TH,
                   int *tx0, int *tx1) {
  if (!v->valid) return 0;
  int ya = ty * TH, yb = ty * TH + TH - 1;
  if (ya < v->y0) ya = v->y0;
  if (yb > v->y1) yb = v->y1;
  if (ya > yb) return 0;
  const float lo = ((float)ya + 0.5f) - v->my;
  const float hi = ((float)yb + 0.5f) - v->my;
  const float dR = fminf(fmaxf(-g->ys, lo), hi);
  const float dL = fminf(fmaxf(g->ys, lo), hi);
  const float at = g->a * g->tau;
  const float eR = g->det * dR;
  const float wR = sqrtf(fmaxf(at - eR * dR, 0.0f));
  const float eL = g->det * dL;
  const float wL = sqrtf(fmaxf(at - eL * dL, 0.0f));
  const float xR = v->mx + ((wR - g->b * dR) * g->ia);
  const float xL = v->mx + ((-wL - g->b * dL) * g->ia);
  const float fx0 = fmaxf(ceilf(xL - 0.5f), v->bx0);
  const float fx1 = fminf(floorf(xR - 0.5f), v->bx1);
  if (!(fx0 <= fx1)) return 0;
  *tx0 = (int)fx0 / TW;
  *tx1 = (int)fx1 / TW;
  return 1;
}

/* Visit the union of the cluster's tiles in ascending tile id. */
typedef void (*tile_cb)(void *ctx, int t);

static int64_t bin_union(int W, int H, int TW, int TH, int C, const float *cq,
                         float tau, const float *means_kc, unsigned char *mark,
                         tile_cb cb, void *ctx) {
  binq g;
  if (!bin_prep(cq[0], cq[1], cq[2], tau, &g)) return 0;
  const int TX = (W + TW - 1) / TW;
  binv vs[256];
  int ty0 = 1 << 30, ty1 = -1;
  const int nv = C < 256 ? C : 256;
  for (int l = 0; l < nv; ++l) {
    bin_view(&g, means_kc[2 * l], means_kc[2 * l + 1], W, H, &vs[l]);
    if (vs[l].valid) {
      if (vs[l].y0 / TH < ty0) ty0 = vs[l].y0 / TH;
      if (vs[l].y1 / TH > ty1) ty1 = vs[l].y1 / TH;
    }
  }
  int64_t n = 0;
  for (int ty = ty0; ty <= ty1; ++ty) {
    int lo = 1 << 30, hi = -1;
    for (int l = 0; l < nv; ++l) {
      int a, b;
      if (!bin_row(&g, &vs[l], ty, TW, TH, &a, &b)) continue;
      for (int tx = a; tx <= b; ++tx) mark[tx] = 1;
      if (a < lo) lo = a;
      if (b > hi) hi = b;
    }
    for (int tx = lo; tx <= hi; ++tx)
      if (mark[tx]) {
        mark[tx] = 0;
        ++n;
        if (cb) cb(ctx, ty * TX + tx);
      }
  }
  return n;
}

int orc_mirror_count(int W, int H, int TW, int TH, int K, int C, int64_t M,
                     const float *conic, const float *tau,
                     const float *mean2d, uint32_t *counts) {
  if (TW <= 0 || TH <= 0 || C <= 0 || C > 256) return -1;
  const int TX = (W + TW - 1) / TW;
#pragma omp parallel
  {
    unsigned char *mark = (unsigned char *)calloc((size_t)TX + 1, 1);
#pragma omp for schedule(dynamic, 256)
    for (int64_t r = 0; r < (int64_t)K * M; ++r)
      counts[r] = (uint32_t)bin_union(W, H, TW, TH, C, conic + 3 * r, tau[r],
                                      mean2d + (size_t)r * C * 2, mark, NULL, NULL);
    free(mark);
  }
  return 0;
}

typedef struct {
  uint64_t *keys;
  uint32_t *vals;
  uint64_t pos;
  uint64_t kbits; /* (k << 32) | depth bits */
  int shift;      /* 32 + Bit_K */
  uint32_t i;
} emit_ctx;

static void emit_cb(void *p, int t) {
  emit_ctx *e = (emit_ctx *)p;
  e->keys[e->pos] = ((uint64_t)t << e->shift) | e->kbits;
  e->vals[e->pos] = e->i;
  e->pos++;
}

static int ceil_log2(uint64_t v) {
  int b = 0;
  while (((uint64_t)1 << b) < v) ++b;
  return b;
}

int orc_mirror_emit(int W, int H, int TW, int TH, int K, int C, int64_t M,
                    const float *conic, const float *tau, const float *depth,
                    const float *mean2d, const uint64_t *offsets,
                    uint64_t *keys, uint32_t *vals) {
  if (TW <= 0 || TH <= 0 || C <= 0 || C > 256) return -1;
  const int TX = (W + TW - 1) / TW;
  const int bit_k = ceil_log2((uint64_t)K);
#pragma omp parallel
  {
    unsigned char *mark = (unsigned char *)calloc((size_t)TX + 1, 1);
#pragma omp for schedule(dynamic, 256)
    for (int64_t r = 0; r < (int64_t)K * M; ++r) {
      const int k = (int)(r / M);
      uint32_t dbits;
      memcpy(&dbits, &depth[r], 4);
      emit_ctx e = {keys, vals, offsets[r], ((uint64_t)k << 32) | dbits, 32 + bit_k,
                    (uint32_t)(r % M)};
      bin_union(W, H, TW, TH, C, conic + 3 * r, tau[r], mean2d + (size_t)r * C * 2, mark,
                emit_cb, &e);
    }
    free(mark);
  }
  return 0;
}

typedef struct {
  uint64_t k;
  uint32_t v;
} kv;

static int cmp_kv(const void *a, const void *b) {
  const kv *x = (const kv *)a, *y = (const kv *)b;
  if (x->k != y->k) return x->k < y->k ? -1 : 1;
  return (x->v > y->v) - (x->v < y->v);
}

int orc_mirror_sort(int64_t P, uint64_t *keys, uint32_t *vals) {
  kv *tmp = (kv *)malloc(sizeof(kv) * (size_t)(P > 0 ? P : 1));
  if (!tmp) return -2;
  for (int64_t p = 0; p < P; ++p) {
    tmp[p].k = keys[p];
    tmp[p].v = vals[p];
  }
  qsort(tmp, (size_t)P, sizeof(kv), cmp_kv);
  for (int64_t p = 0; p < P; ++p) {
    keys[p] = tmp[p].k;
    vals[p] = tmp[p].v;
  }
  free(tmp);
  return 0;
}

int orc_mirror_ranges(int64_t P, const uint64_t *keys_sorted, int bit_k,
                      int T, int K, uint32_t *ranges) {
  memset(ranges, 0, sizeof(uint32_t) * 2 * (size_t)T * K);
  for (int64_t p = 0; p < P; ++p) {
    const uint64_t tk = keys_sorted[p] >> 32;
    const uint64_t t = tk >> bit_k, k = tk & (((uint64_t)1 << bit_k) - 1);
    if (t >= (uint64_t)T || k >= (uint64_t)K) return -1;
    const size_t s = (size_t)(t * K + k);
    if (p == 0 || (keys_sorted[p - 1] >> 32) != tk) ranges[2 * s] = (uint32_t)p;
    if (p == P - 1 || (keys_sorted[p + 1] >> 32) != tk) ranges[2 * s + 1] = (uint32_t)(p + 1);
  }
  return 0;
}
