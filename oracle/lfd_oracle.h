/*
 * Plain CPU oracle for subpixel-level 3DGS rasterisation of an interlaced
 * light-field image (CoherentRaster, arXiv 2605.04509).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call, link or
 * load this code; it is used by the tests, by the smoke check and by the CPU
 * baseline leg of the benchmark. It shares no code with the CUDA library.
 *
 * Floating point is FP64 everywhere the paper leaves precision open, except
 * the "mirror" functions (orc_mirror_*), which take the integer decisions of
 * the GPU path (tile bins) in the kernel's precision, FP32, with every
 * operation correctly rounded and no contraction, so that tile bins, keys,
 * the sorted list and the range table can be compared bit for bit.
 *
 * Conventions shared with the CUDA path only through their definitions:
 *   cameras   float32 [N][16]: R (row-major world->camera), t, fx, fy, cx, cy
 *   V         uint8 [H][W][3] view index per subpixel (x, y, u)
 *   psi       uint16 per tile, tile-major, stride TW*TH*3: local row-major
 *             subpixel index (yl*TW + xl)*3 + u, sorted stably by view
 *   seg       int32 [T][K+1] start of each cluster's run inside psi
 *   clusters  slot l of cluster k is view min(k*C + l, N-1); the
 *             representative is view min(k*C + floor(C/2), N-1)
 */
#ifndef LFD_ORACLE_H
#define LFD_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Eq. 1-3: view index of every subpixel. Returns 0, or -1 on bad input. */
int orc_view_index(int W, int H, int N, double tan_slant, double pitch,
                   double k_offset, uint8_t *V);

/* Sec. 4.3, Eq. 8: per-tile stable sort of row-major subpixels by view. */
int orc_remap(int W, int H, int N, const uint8_t *V, int TW, int TH, int C,
              uint16_t *psi, int32_t *n_sub, int32_t *seg);

/* Appendix B.1: contiguous clusters padded with the last view. */
int orc_clusters(int N, int C, int32_t *slot_view, int32_t *rep);

/* Eq. 4-6 in FP64. Outputs: per-view means [N][M][2] and validity [N][M];
 * per-cluster conic [K][M][3], depth [K][M], colour [K][M][3],
 * tau = 2 ln(255 o) [K][M] and validity [K][M]. The depth (and the
 * near-plane test z > 0.2) is the one FP32 quantity: Eq. 11 keys order by the
 * bits of a 32-bit float depth, so it is evaluated as
 * ((R20 mx + R21 my) + R22 mz) + t2 with every operation rounded to float. */
int orc_project(int64_t M, const float *means, const float *scales,
                const float *quats, const float *opac, const float *sh,
                int sh_degree, int N, const float *cams, int W, int H, int C,
                double *mean2d, uint8_t *vvalid, double *conic, double *depth,
                double *color, double *tau, uint8_t *valid);

/* Eq. 9-10 with the 3DGS rules, per subpixel of the crop [x0,x1)x[y0,y1).
 * mode 0: walk every valid Gaussian of the subpixel's cluster in (depth, id)
 * order (the definition); mode 1: the same walk restricted to per-(tile,
 * cluster) lists built from conservative bounding boxes (same result).
 * out is [(y1-y0)][(x1-x0)][3]; n_eval (nullable) counts visited entries. */
int orc_render(int W, int H, int N, int C, const uint8_t *V, int TW, int TH,
               int64_t M, const double *mean2d, const uint8_t *vvalid,
               const double *conic, const double *depth, const double *color,
               const uint8_t *valid, const double *opac, int x0, int y0,
               int x1, int y1, int mode, const double *bg, double *out,
               int64_t *n_eval);

/* The same blend along explicitly given lists: ranges [T][K][2] into list. */
int orc_blend_lists(int W, int H, int N, int C, const uint8_t *V, int TW,
                    int TH, int64_t M, const double *mean2d,
                    const uint8_t *vvalid, const double *conic,
                    const double *color, const double *opac,
                    const uint32_t *ranges, const uint32_t *list, int x0,
                    int y0, int x1, int y1, const double *bg, double *out,
                    int64_t *n_eval);

/* Full-frame 3DGS of every view followed by interlacing (Sec. 1, Sec. 5.1
 * baseline). Attributes are per view (a projection with C = 1). */
int orc_render_fullframe(int W, int H, int N, const uint8_t *V, int64_t M,
                         const double *mean2d, const uint8_t *vvalid,
                         const double *conic, const double *depth,
                         const double *color, const uint8_t *valid,
                         const double *opac, int x0, int y0, int x1, int y1,
                         const double *bg, double *out);

/* FP32 mirror of the tile-bin rule (Alg. 2 GenerateKeys): tile count of the
 * union over the cluster's views, per (k, i). Inputs are float32:
 * conic [K][M][3], tau [K][M], mean2d [K][M][C][2] (cluster slots; a
 * non-finite mean marks a view in which the Gaussian is culled). */
int orc_mirror_count(int W, int H, int TW, int TH, int K, int C, int64_t M,
                     const float *conic, const float *tau,
                     const float *mean2d, uint32_t *counts);

/* Emission of Eq. 11 keys in (k, i) order at the given offsets. */
int orc_mirror_emit(int W, int H, int TW, int TH, int K, int C, int64_t M,
                    const float *conic, const float *tau, const float *depth,
                    const float *mean2d, const uint64_t *offsets,
                    uint64_t *keys, uint32_t *vals);

/* Ascending sort of (key, value) pairs; equal keys keep ascending values. */
int orc_mirror_sort(int64_t P, uint64_t *keys, uint32_t *vals);

/* Range table [T][K][2] = [S, E) of each (tile, cluster) list. */
int orc_mirror_ranges(int64_t P, const uint64_t *keys_sorted, int bit_k,
                      int T, int K, uint32_t *ranges);

/* Set the alpha skip threshold used by the blends (default 1/255, the 3DGS
 * rule) and return the previous one; v <= 0 leaves it unchanged. The
 * definition is discontinuous at this threshold: tests render it slightly
 * above and below to find the subpixels where the result itself jumps. */
double orc_set_alpha_min(double v);

int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
