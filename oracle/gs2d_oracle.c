/*
 * gs2d_oracle.c -- FP64 CPU oracle of the 2D Gaussian (surfel) splatting
 * rasterizer used by CityGaussianV2 (arXiv 2411.00771).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow definition that the
 * CUDA path is checked against.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant generator with the CUDA library.
 *
 * Passages followed (section / equation of the paper):
 *   - Eq. 1 (Sec. 3.1): front-to-back alpha compositing over the primitives on
 *     a pixel's ray, alpha = opacity * Gaussian falloff.
 *   - Sec. 3.1 "2D Gaussian Splatting": a surfel is a disk with tangents t_u,
 *     t_v and scales (s_u, s_v); normal = t_u x t_v; depth distortion and
 *     normal terms are rendered alongside colour.
 *   - Sec. 3.2 (elongation filter paragraph): sub-pixel splats are handled by
 *     the antialiasing low-pass filter (object/screen-space max).
 *   - Sec. 5.1: median depth is rendered for geometry.
 *   - Sec. 3.1: L1 + D-SSIM photometric loss; Sec. 3.2: depth loss on inverse
 *     depth; Sec. 3.2 Eq. 2: decomposed-gradient densification; Sec. 3.2:
 *     elongation rate eta = min(s)/max(s).
 *   - Sec. 3.3 Eq. 3: single-view trim contribution of each surfel.
 *   - Sec. 4: visible frequency of points (crop volume estimation).
 * Readings where the paper is silent (pixel centres at +0.5, alpha clamp 0.99,
 * stop before the pair that would take T below T_min, the per-pair 3-sigma
 * support rho <= 9, screen filter rho_scr = 2 |x - c|^2, centre depth when the
 * screen filter wins, median = last blended pair entered with T > 0.5, the
 * compositing order key = centre depth rounded to FP32 with ties by index)
 * are the ones listed in the design notes of this repository.
 *
 * Everything is double precision.  Inputs are double arrays; the tests pass
 * the FP32 values the CUDA path receives, widened exactly to double.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- camera and settings arrays (marshalled from Python as doubles) ---- */
enum { CAM_R = 0, CAM_T = 9, CAM_FX = 12, CAM_FY = 13, CAM_CX = 14, CAM_CY = 15,
       CAM_W = 16, CAM_H = 17, CAM_LEN = 18 };
enum { SET_NEAR = 0, SET_ALPHA_MIN = 1, SET_T_MIN = 2, SET_ALPHA_MAX = 3,
       SET_RHO_MAX = 4, SET_SCREEN_INV_S2 = 5, SET_BG = 6 /* 3 values */,
       SET_TILE = 9, SET_LEN = 10 };

/* output planes of a render, [OUT_PLANES][H][W] */
enum { O_R = 0, O_G = 1, O_B = 2, O_ALPHA = 3, O_DEPTH = 4, O_INVDEPTH = 5,
       O_MEDIAN = 6, O_NX = 7, O_NY = 8, O_NZ = 9, O_DIST = 10, O_TFINAL = 11,
       OUT_PLANES = 12, ADJ_PLANES = 11 };

/* per-pixel flags: a decision taken within a hair of a threshold.  The
 * margins (relative 1e-5 for alpha, the transmittance stop and the median
 * pivot; 1e-4 absolute on rho) exceed the FP32 error of those quantities
 * after tens of compositing steps (a few 1e-7 relative). */
enum { F_ALPHA = 1, F_RHO = 2, F_TSTOP = 4, F_MEDIAN = 8, F_BRANCH = 16 };

typedef struct {
  double M[9];      /* homography K [R_c s_u t_u | R_c s_v t_v | p_c], row-major */
  double rgb[3];
  double nrm[3];    /* view-space normal facing the camera */
  double opac;
  double zkey;      /* centre depth rounded to FP32 (order key) */
  double bbox[4];   /* xmin xmax ymin ymax of the 3-sigma cover, pixels */
  int rect[4];      /* tile rect [tx0, ty0, tx1, ty1) */
  int live;         /* not culled */
  double rawcol[3]; /* SH sum + 0.5 before the clamp */
  double cond;      /* condition number of the centred 2x2 Jacobian */
  /* footprint shape for per-row tile coverage: ellipse {rho_obj <= rho_max}
   * with centre e0 and matrix G ((x - e0)^T G^-1 (x - e0) <= 1), screen disk
   * centre sc and radius rf, pixel-centre index box [ilo, ihi] x [jlo, jhi] */
  double e0[2], G[3], sc[2], rf;
  int pix[4];
  int ntiles;       /* tiles the footprint reaches (per-row rule) */
  int rownear;      /* a row interval end within 1e-6 px of a pixel-centre boundary */
} pre_t;

typedef struct {
  int n;
  int obj;          /* 1: object-space branch won */
  double x, y;
  double u, v, h[3], l1[3], l2[3];
  double rho, rho_obj, rho_scr, G, araw, alpha, z;
  double T;         /* transmittance before this pair */
  double w;
} pair_t;

/* ---------------------------------------------------------------------- */
/* Real spherical harmonics, degree <= 3, Condon-Shortley phase kept, index
 * k = l*l + l + m.  Written from the Cartesian forms of the real basis; the
 * orthonormality and the match with the complex basis are checked in tests. */
static void sh_basis(const double d[3], double Y[16], double dY[16][3]) {
  const double x = d[0], y = d[1], z = d[2];
  const double pi = 3.14159265358979323846;
  const double c0 = 0.5 / sqrt(pi);
  const double c1 = sqrt(3.0 / (4.0 * pi));
  const double c2a = 0.5 * sqrt(15.0 / pi);
  const double c2b = 0.25 * sqrt(5.0 / pi);
  const double c2c = 0.25 * sqrt(15.0 / pi);
  const double c3a = 0.25 * sqrt(35.0 / (2.0 * pi));
  const double c3b = 0.5 * sqrt(105.0 / pi);
  const double c3c = 0.25 * sqrt(21.0 / (2.0 * pi));
  const double c3d = 0.25 * sqrt(7.0 / pi);
  const double c3e = 0.25 * sqrt(105.0 / pi);
  double g[16][3];
  memset(g, 0, sizeof g);
  Y[0] = c0;
  Y[1] = -c1 * y;           g[1][1] = -c1;
  Y[2] = c1 * z;            g[2][2] = c1;
  Y[3] = -c1 * x;           g[3][0] = -c1;
  Y[4] = c2a * x * y;       g[4][0] = c2a * y; g[4][1] = c2a * x;
  Y[5] = -c2a * y * z;      g[5][1] = -c2a * z; g[5][2] = -c2a * y;
  Y[6] = c2b * (2 * z * z - x * x - y * y);
  g[6][0] = -2 * c2b * x; g[6][1] = -2 * c2b * y; g[6][2] = 4 * c2b * z;
  Y[7] = -c2a * x * z;      g[7][0] = -c2a * z; g[7][2] = -c2a * x;
  Y[8] = c2c * (x * x - y * y); g[8][0] = 2 * c2c * x; g[8][1] = -2 * c2c * y;
  Y[9] = -c3a * y * (3 * x * x - y * y);
  g[9][0] = -c3a * 6 * x * y; g[9][1] = -c3a * (3 * x * x - 3 * y * y);
  Y[10] = c3b * x * y * z;
  g[10][0] = c3b * y * z; g[10][1] = c3b * x * z; g[10][2] = c3b * x * y;
  Y[11] = -c3c * y * (4 * z * z - x * x - y * y);
  g[11][0] = -c3c * (-2 * x * y); g[11][1] = -c3c * (4 * z * z - x * x - 3 * y * y);
  g[11][2] = -c3c * 8 * y * z;
  Y[12] = c3d * z * (2 * z * z - 3 * x * x - 3 * y * y);
  g[12][0] = c3d * (-6 * x * z); g[12][1] = c3d * (-6 * y * z);
  g[12][2] = c3d * (6 * z * z - 3 * x * x - 3 * y * y);
  Y[13] = -c3c * x * (4 * z * z - x * x - y * y);
  g[13][0] = -c3c * (4 * z * z - 3 * x * x - y * y); g[13][1] = -c3c * (-2 * x * y);
  g[13][2] = -c3c * 8 * x * z;
  Y[14] = c3e * z * (x * x - y * y);
  g[14][0] = c3e * 2 * x * z; g[14][1] = -c3e * 2 * y * z; g[14][2] = c3e * (x * x - y * y);
  Y[15] = -c3a * x * (x * x - 3 * y * y);
  g[15][0] = -c3a * (3 * x * x - 3 * y * y); g[15][1] = -c3a * (-6 * x * y);
  if (dY) memcpy(dY, g, sizeof g);
}

/* exported for the basis pins */
void oracle_sh_basis(int n, const double* dirs, double* Y) {
  for (int i = 0; i < n; ++i) sh_basis(dirs + 3 * i, Y + 16 * i, NULL);
}

/* Rotation matrix of a unit quaternion (w, x, y, z), row-major. */
static void quat_to_R(const double q[4], double R[9]) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y); R[7] = 2 * (y * z + w * x); R[8] = 1 - 2 * (x * x + y * y);
}

/* dL/dq for R(q) given G = dL/dR (row-major), q unit (w,x,y,z). */
static void quat_to_R_vjp(const double q[4], const double G[9], double dq[4]) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  /* partial derivatives of every entry, written from the formula above */
  const double dRw[9] = {0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0};
  const double dRx[9] = {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x};
  const double dRy[9] = {-4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y};
  const double dRz[9] = {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0};
  dq[0] = dq[1] = dq[2] = dq[3] = 0;
  for (int i = 0; i < 9; ++i) {
    dq[0] += G[i] * dRw[i]; dq[1] += G[i] * dRx[i];
    dq[2] += G[i] * dRy[i]; dq[3] += G[i] * dRz[i];
  }
}

static void cross3(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static void matvec3(const double R[9], const double v[3], double o[3]) {
  for (int i = 0; i < 3; ++i) o[i] = R[3 * i] * v[0] + R[3 * i + 1] * v[1] + R[3 * i + 2] * v[2];
}
static void matTvec3(const double R[9], const double v[3], double o[3]) {
  for (int i = 0; i < 3; ++i) o[i] = R[i] * v[0] + R[3 + i] * v[1] + R[6 + i] * v[2];
}

typedef struct {
  int64_t N;
  int deg, K;
  const double *mu, *quat, *scale, *opac, *sh;
} scene_t;

static void cam_pos(const double* cam, double o[3]) {
  /* camera centre in world = -R^T t */
  double mt[3];
  matTvec3(cam + CAM_R, cam + CAM_T, mt);
  o[0] = -mt[0]; o[1] = -mt[1]; o[2] = -mt[2];
}

/* ---------------------------------------------------------------------- */
/* Tile coverage of one row of tiles.  The footprint {rho <= rho_max} is the
 * union of the projected disk (an ellipse, centre e0, matrix G) and the
 * screen-filter disk.  Over the band of pixel-centre rows of tile row ty,
 * each convex part spans an x interval: the ellipse's x(y) on its right
 * boundary is concave, so its largest value over the band is at the
 * rightmost point's y clamped to the band (the leftmost likewise); the
 * disk's widest point is at its centre's y clamped to the band.  The tiles
 * of the pixel centres inside the hull of the two intervals are covered.
 * Returns 0 when the row is empty, else the tile columns [tx0, tx1). */
static int row_tiles(pre_t* P, int ty, int tile, int* tx0, int* tx1) {
  int ja = ty * tile, jb = ty * tile + tile - 1;
  if (ja < P->pix[2]) ja = P->pix[2];
  if (jb > P->pix[3]) jb = P->pix[3];
  if (ja > jb) return 0;
  const double ya = ja + 0.5, yb = jb + 0.5;
  double lo = INFINITY, hi = -INFINITY;
  const double g11 = P->G[0], g12 = P->G[1], g22 = P->G[2];
  if (g11 > 0 && g22 > 0) {
    const double hx = sqrt(g11), hy = sqrt(g22);
    const double dya = ya - P->e0[1], dyb = yb - P->e0[1];
    if (dyb >= -hy && dya <= hy) {
      const double det = fmax(g11 * g22 - g12 * g12, 0.0);
      /* rightmost point at dy = g12 / hx, leftmost at -g12 / hx */
      double yr = g12 / hx, yl = -g12 / hx;
      yr = yr < dya ? dya : (yr > dyb ? dyb : yr);
      yl = yl < dya ? dya : (yl > dyb ? dyb : yl);
      hi = P->e0[0] + (g12 * yr + sqrt(fmax(det * (g22 - yr * yr), 0.0))) / g22;
      lo = P->e0[0] + (g12 * yl - sqrt(fmax(det * (g22 - yl * yl), 0.0))) / g22;
    }
  }
  double yn = P->sc[1];
  yn = yn < ya ? ya : (yn > yb ? yb : yn);
  const double dy = yn - P->sc[1];
  if (dy * dy <= P->rf * P->rf) {
    const double h = sqrt(P->rf * P->rf - dy * dy);
    if (P->sc[0] - h < lo) lo = P->sc[0] - h;
    if (P->sc[0] + h > hi) hi = P->sc[0] + h;
  }
  if (!(lo <= hi)) return 0;
  if (fabs((lo - 0.5) - nearbyint(lo - 0.5)) < 1e-6 || fabs((hi - 0.5) - nearbyint(hi - 0.5)) < 1e-6)
    P->rownear = 1;
  double ilo = ceil(lo - 0.5), ihi = floor(hi - 0.5);
  if (ilo < P->pix[0]) ilo = P->pix[0];
  if (ihi > P->pix[1]) ihi = P->pix[1];
  if (ilo > ihi) return 0;
  *tx0 = (int)ilo / tile;
  *tx1 = (int)ihi / tile + 1;
  return 1;
}

/* ---------------------------------------------------------------------- */
/* Per-surfel preprocess: the definition's steps 1-3, 7, 8 and the 3-sigma
 * cover (conic bounding box) plus the screen-filter disc. */
static void preprocess_one(const scene_t* S, int64_t n, const double* cam,
                           const double* set, pre_t* P) {
  memset(P, 0, sizeof *P);
  const double* Rc = cam + CAM_R;
  const double* tc = cam + CAM_T;
  const double fx = cam[CAM_FX], fy = cam[CAM_FY], cx = cam[CAM_CX], cy = cam[CAM_CY];
  const int W = (int)cam[CAM_W], H = (int)cam[CAM_H];
  const int tile = (int)set[SET_TILE];
  double q[4] = {S->quat[4 * n], S->quat[4 * n + 1], S->quat[4 * n + 2], S->quat[4 * n + 3]};
  double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  if (!(qn > 0)) return;
  for (int i = 0; i < 4; ++i) q[i] /= qn;
  double R[9];
  quat_to_R(q, R);
  const double r1[3] = {R[0], R[3], R[6]}, r2[3] = {R[1], R[4], R[7]}, r3[3] = {R[2], R[5], R[8]};
  const double mu[3] = {S->mu[3 * n], S->mu[3 * n + 1], S->mu[3 * n + 2]};
  const double su = S->scale[2 * n], sv = S->scale[2 * n + 1];
  double p[3], tu[3], tv[3], nv[3];
  matvec3(Rc, mu, p);
  for (int i = 0; i < 3; ++i) p[i] += tc[i];
  matvec3(Rc, r1, tu);
  matvec3(Rc, r2, tv);
  matvec3(Rc, r3, nv);
  const double a[3] = {su * tu[0], su * tu[1], su * tu[2]};
  const double b[3] = {sv * tv[0], sv * tv[1], sv * tv[2]};
  /* cull: the 3-sigma disc must lie entirely beyond the near plane */
  const double sig = sqrt(set[SET_RHO_MAX]);
  const double zmin = p[2] - sig * sqrt(a[2] * a[2] + b[2] * b[2]);
  if (!(zmin > set[SET_NEAR])) return;
  double* M = P->M;
  M[0] = fx * a[0] + cx * a[2]; M[1] = fx * b[0] + cx * b[2]; M[2] = fx * p[0] + cx * p[2];
  M[3] = fy * a[1] + cy * a[2]; M[4] = fy * b[1] + cy * b[2]; M[5] = fy * p[1] + cy * p[2];
  M[6] = a[2];                  M[7] = b[2];                  M[8] = p[2];
  P->live = 1;
  P->opac = S->opac[n];
  P->zkey = (double)(float)p[2];
  /* normal facing the camera */
  const double sgn = dot3(nv, p) > 0 ? -1.0 : 1.0;
  for (int i = 0; i < 3; ++i) P->nrm[i] = sgn * nv[i];
  /* colour from SH, world direction from camera centre to mu */
  double o[3], d[3];
  cam_pos(cam, o);
  for (int i = 0; i < 3; ++i) d[i] = mu[i] - o[i];
  const double dl = sqrt(dot3(d, d));
  for (int i = 0; i < 3; ++i) d[i] /= dl;
  double Y[16];
  sh_basis(d, Y, NULL);
  for (int c = 0; c < 3; ++c) {
    double acc = 0;
    for (int k = 0; k < S->K; ++k) acc += S->sh[(n * S->K + k) * 3 + c] * Y[k];
    P->rawcol[c] = acc + 0.5;
    P->rgb[c] = P->rawcol[c] > 0 ? P->rawcol[c] : 0.0;
  }
  /* bounding box of {rho_obj <= rho_max}: dual conic C* = M diag(r,r,-1) M^T,
   * vertical tangents solve C*11 - 2 x C*13 + x^2 C*33 = 0 */
  const double r = set[SET_RHO_MAX];
  const double C11 = r * (M[0] * M[0] + M[1] * M[1]) - M[2] * M[2];
  const double C22 = r * (M[3] * M[3] + M[4] * M[4]) - M[5] * M[5];
  const double C13 = r * (M[0] * M[6] + M[1] * M[7]) - M[2] * M[8];
  const double C23 = r * (M[3] * M[6] + M[4] * M[7]) - M[5] * M[8];
  const double C33 = r * (M[6] * M[6] + M[7] * M[7]) - M[8] * M[8];
  const double C12 = r * (M[0] * M[3] + M[1] * M[4]) - M[2] * M[5];
  /* the dual conic scaled to C*33 = 1 is [[e0 e0^T - G, e0], [e0^T, 1]] for
   * the ellipse (x - e0)^T G^-1 (x - e0) <= 1: centre and shape directly */
  P->e0[0] = C13 / C33;
  P->e0[1] = C23 / C33;
  P->G[0] = P->e0[0] * P->e0[0] - C11 / C33;
  P->G[1] = P->e0[0] * P->e0[1] - C12 / C33;
  P->G[2] = P->e0[1] * P->e0[1] - C22 / C33;
  double dx = C13 * C13 - C11 * C33, dy = C23 * C23 - C22 * C33;
  dx = dx > 0 ? sqrt(dx) : 0; dy = dy > 0 ? sqrt(dy) : 0;
  double x0 = (C13 - dx) / C33, x1 = (C13 + dx) / C33;
  double y0 = (C23 - dy) / C33, y1 = (C23 + dy) / C33;
  double xmin = fmin(x0, x1), xmax = fmax(x0, x1), ymin = fmin(y0, y1), ymax = fmax(y0, y1);
  const double ccx = M[2] / M[8], ccy = M[5] / M[8];
  const double rf = sqrt(set[SET_RHO_MAX] / set[SET_SCREEN_INV_S2]);
  xmin = fmin(xmin, ccx - rf); xmax = fmax(xmax, ccx + rf);
  ymin = fmin(ymin, ccy - rf); ymax = fmax(ymax, ccy + rf);
  P->bbox[0] = xmin; P->bbox[1] = xmax; P->bbox[2] = ymin; P->bbox[3] = ymax;
  /* pixels whose centre (i + 0.5) lies inside the box */
  double ilo = ceil(xmin - 0.5), ihi = floor(xmax - 0.5);
  double jlo = ceil(ymin - 0.5), jhi = floor(ymax - 0.5);
  if (ilo < 0) ilo = 0;
  if (jlo < 0) jlo = 0;
  if (ihi > W - 1) ihi = W - 1;
  if (jhi > H - 1) jhi = H - 1;
  P->sc[0] = ccx; P->sc[1] = ccy; P->rf = rf;
  if (ilo > ihi || jlo > jhi) {
    P->rect[0] = P->rect[1] = P->rect[2] = P->rect[3] = 0;
  } else {
    P->rect[0] = (int)ilo / tile; P->rect[1] = (int)jlo / tile;
    P->rect[2] = (int)ihi / tile + 1; P->rect[3] = (int)jhi / tile + 1;
    P->pix[0] = (int)ilo; P->pix[1] = (int)ihi; P->pix[2] = (int)jlo; P->pix[3] = (int)jhi;
    for (int ty = P->rect[1]; ty < P->rect[3]; ++ty) {
      int a, b;
      if (row_tiles(P, ty, tile, &a, &b)) P->ntiles += b - a;
    }
  }
  /* condition number of the centred Jacobian d(offset)/d(u,v) at the centre:
   * used only to flag pixels whose FP32 evaluation is ill-conditioned */
  const double J11 = fx * (a[0] - a[2] * p[0] / p[2]) / p[2];
  const double J12 = fx * (b[0] - b[2] * p[0] / p[2]) / p[2];
  const double J21 = fy * (a[1] - a[2] * p[1] / p[2]) / p[2];
  const double J22 = fy * (b[1] - b[2] * p[1] / p[2]) / p[2];
  const double fro2 = J11 * J11 + J12 * J12 + J21 * J21 + J22 * J22;
  const double det = fabs(J11 * J22 - J12 * J21);
  /* sigma_max / sigma_min = (f + sqrt(f^2 - 4 det^2)) / (2 det) with f = ||J||_F^2 */
  const double disc = sqrt(fmax(fro2 * fro2 - 4 * det * det, 0.0));
  P->cond = det > 0 ? (fro2 + disc) / (2 * det) : INFINITY;
}

/* Evaluate surfel n at pixel sample (x, y): steps 4-6 of the definition. */
static void eval_pair(const pre_t* P, int n, double x, double y, const double* set, pair_t* pr) {
  const double* M = P->M;
  pr->n = n; pr->x = x; pr->y = y;
  const double m1[3] = {M[0], M[1], M[2]}, m2[3] = {M[3], M[4], M[5]}, m3[3] = {M[6], M[7], M[8]};
  for (int i = 0; i < 3; ++i) { pr->l1[i] = m1[i] - x * m3[i]; pr->l2[i] = m2[i] - y * m3[i]; }
  cross3(pr->l1, pr->l2, pr->h);
  double zobj = 0;
  if (pr->h[2] != 0) {
    pr->u = pr->h[0] / pr->h[2];
    pr->v = pr->h[1] / pr->h[2];
    pr->rho_obj = pr->u * pr->u + pr->v * pr->v;
    zobj = m3[0] * pr->u + m3[1] * pr->v + m3[2];
  } else {
    pr->u = pr->v = 0;
    pr->rho_obj = INFINITY;
  }
  const double ccx = M[2] / M[8], ccy = M[5] / M[8];
  pr->rho_scr = set[SET_SCREEN_INV_S2] * ((x - ccx) * (x - ccx) + (y - ccy) * (y - ccy));
  if (pr->rho_obj <= pr->rho_scr) { pr->obj = 1; pr->rho = pr->rho_obj; pr->z = zobj; }
  else { pr->obj = 0; pr->rho = pr->rho_scr; pr->z = M[8]; }
  pr->G = exp(-0.5 * pr->rho);
  pr->araw = P->opac * pr->G;
  pr->alpha = pr->araw < set[SET_ALPHA_MAX] ? pr->araw : set[SET_ALPHA_MAX];
}

typedef struct {
  double out[OUT_PLANES];
  double dexact;
  int count;
  int flags;
  int ncand;
} pix_t;

/* sort key context: zkey per surfel */
typedef struct { double z; int n; int slot; } okey_t;
static int cmp_keys(const void* A, const void* B) {
  const okey_t* a = (const okey_t*)A;
  const okey_t* b = (const okey_t*)B;
  if (a->z < b->z) return -1;
  if (a->z > b->z) return 1;
  return (a->n > b->n) - (a->n < b->n);
}

/* Composite one pixel over a candidate index list (brute force: every live
 * surfel; binned: the pixel's tile list).  Fills the blended pairs in order
 * into `blended` (capacity cap) and the per-pixel outputs. */
/* rho = min(rho_obj, rho_scr) of surfel P at pixel sample (x, y). */
static double eval_rho(const pre_t* P, double x, double y, const double* set) {
  pair_t pr;
  eval_pair(P, 0, x, y, set, &pr);
  return pr.rho;
}

static int composite_pixel(const pre_t* pre, const int* cand, int ncand, double x, double y,
                           const double* set, const double* shift, pair_t* tmp, okey_t* keys,
                           pair_t* blended, pix_t* px) {
  memset(px, 0, sizeof *px);
  int m = 0;
  for (int c = 0; c < ncand; ++c) {
    const int n = cand[c];
    if (!pre[n].live) continue;
    pair_t pr;
    eval_pair(&pre[n], n, x, y, set, &pr);
    if (shift) {
      /* footprint translated by delta_n on screen: the opacity falloff is
       * evaluated at x - delta_n; colour, depth and normal stay as they are
       * (definition of the screen-space densification gradient) */
      pr.rho = eval_rho(&pre[n], x - shift[2 * n], y - shift[2 * n + 1], set);
      pr.G = exp(-0.5 * pr.rho);
      pr.araw = pre[n].opac * pr.G;
      pr.alpha = pr.araw < set[SET_ALPHA_MAX] ? pr.araw : set[SET_ALPHA_MAX];
    }
    if (!(pr.rho <= set[SET_RHO_MAX])) {
      if (fabs(pr.rho - set[SET_RHO_MAX]) < 1e-4) px->flags |= F_RHO;
      continue;
    }
    if (fabs(pr.rho - set[SET_RHO_MAX]) < 1e-4) px->flags |= F_RHO;
    if (fabs(pr.alpha / set[SET_ALPHA_MIN] - 1.0) < 1e-5) px->flags |= F_ALPHA;
    if (!(pr.alpha >= set[SET_ALPHA_MIN])) continue;
    tmp[m] = pr;
    keys[m].z = pre[n].zkey; keys[m].n = n; keys[m].slot = m;
    ++m;
  }
  px->ncand = m;
  qsort(keys, (size_t)m, sizeof(okey_t), cmp_keys);
  double T = 1.0, A = 0, Z = 0;
  int nb = 0;
  for (int k = 0; k < m; ++k) {
    pair_t pr = tmp[keys[k].slot];
    const double Tn = T * (1.0 - pr.alpha);
    if (fabs(Tn / set[SET_T_MIN] - 1.0) < 1e-5) px->flags |= F_TSTOP;
    if (Tn < set[SET_T_MIN]) break;
    const double w = pr.alpha * T;
    pr.T = T; pr.w = w;
    const pre_t* P = &pre[pr.n];
    for (int c = 0; c < 3; ++c) px->out[O_R + c] += w * P->rgb[c];
    px->out[O_DIST] += 2.0 * w * (pr.z * A - Z);
    A += w;
    Z += w * pr.z;
    px->out[O_INVDEPTH] += w / pr.z;
    for (int c = 0; c < 3; ++c) px->out[O_NX + c] += w * P->nrm[c];
    if (fabs(T / 0.5 - 1.0) < 1e-5) px->flags |= F_MEDIAN;
    if (T > 0.5) px->out[O_MEDIAN] = pr.z;
    if (pr.obj && fabs(pr.rho_obj - pr.rho_scr) < 1e-5 * (1 + pr.rho_scr)) px->flags |= F_BRANCH;
    blended[nb++] = pr;
    T = Tn;
  }
  px->out[O_ALPHA] = A;
  px->out[O_DEPTH] = Z;
  px->out[O_TFINAL] = T;
  for (int c = 0; c < 3; ++c) px->out[O_R + c] += T * set[SET_BG + c];
  px->count = nb;
  double de = 0;
  for (int i = 0; i < nb; ++i)
    for (int j = 0; j < nb; ++j) de += blended[i].w * blended[j].w * fabs(blended[i].z - blended[j].z);
  px->dexact = de;
  return nb;
}

/* ---------------------------------------------------------------------- */
/* Public entry points (ctypes).                                           */

static scene_t mk_scene(int64_t N, int deg, const double* mu, const double* quat, const double* scale,
                        const double* opac, const double* sh) {
  scene_t S;
  S.N = N; S.deg = deg; S.K = (deg + 1) * (deg + 1);
  S.mu = mu; S.quat = quat; S.scale = scale; S.opac = opac; S.sh = sh;
  return S;
}

/* Preprocess: per surfel M[9], rgb[3], normal[3], zkey, bbox[4], rect[4],
 * live flag, the Jacobian condition number, the number of tiles the
 * footprint reaches (per-row rule) and whether a row interval ends within
 * 1e-6 px of a pixel-centre boundary. */
int oracle_preprocess(int64_t N, int deg, const double* mu, const double* quat, const double* scale,
                      const double* opac, const double* sh, const double* cam, const double* set,
                      double* M, double* rgb, double* nrm, double* zkey, double* bbox, int* rect,
                      int* live, double* cond, int* ntiles, int* rownear) {
  scene_t S = mk_scene(N, deg, mu, quat, scale, opac, sh);
#pragma omp parallel for schedule(static)
  for (int64_t n = 0; n < N; ++n) {
    pre_t P;
    preprocess_one(&S, n, cam, set, &P);
    memcpy(M + 9 * n, P.M, sizeof P.M);
    memcpy(rgb + 3 * n, P.rgb, sizeof P.rgb);
    memcpy(nrm + 3 * n, P.nrm, sizeof P.nrm);
    zkey[n] = P.zkey;
    memcpy(bbox + 4 * n, P.bbox, sizeof P.bbox);
    memcpy(rect + 4 * n, P.rect, sizeof P.rect);
    live[n] = P.live;
    cond[n] = P.cond;
    if (ntiles) ntiles[n] = P.live ? P.ntiles : 0;
    if (rownear) rownear[n] = P.rownear;
  }
  return 0;
}

/* Tile lists: for each tile, surfels (by index) whose rect covers it. */
typedef struct { int64_t* start; int* idx; int ntiles; int tile; } tiles_t;

static void build_tiles(const pre_t* pre, int64_t N, int tx, int ty, tiles_t* T) {
  T->ntiles = tx * ty;
  T->start = (int64_t*)calloc((size_t)T->ntiles + 1, sizeof(int64_t));
  const int tile = (int)(T->tile);
  for (int64_t n = 0; n < N; ++n) {
    if (!pre[n].live) continue;
    pre_t P = pre[n];
    for (int j = P.rect[1]; j < P.rect[3]; ++j) {
      int a, b;
      if (!row_tiles(&P, j, tile, &a, &b)) continue;
      for (int i = a; i < b; ++i) T->start[j * tx + i + 1]++;
    }
  }
  for (int t = 0; t < T->ntiles; ++t) T->start[t + 1] += T->start[t];
  T->idx = (int*)malloc(sizeof(int) * (size_t)(T->start[T->ntiles] + 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)T->ntiles);
  memcpy(fill, T->start, sizeof(int64_t) * (size_t)T->ntiles);
  for (int64_t n = 0; n < N; ++n) {
    if (!pre[n].live) continue;
    pre_t P = pre[n];
    for (int j = P.rect[1]; j < P.rect[3]; ++j) {
      int a, b;
      if (!row_tiles(&P, j, tile, &a, &b)) continue;
      for (int i = a; i < b; ++i) T->idx[fill[j * tx + i]++] = (int)n;
    }
  }
  free(fill);
}

static pre_t* run_preprocess(const scene_t* S, const double* cam, const double* set) {
  pre_t* pre = (pre_t*)malloc(sizeof(pre_t) * (size_t)(S->N > 0 ? S->N : 1));
#pragma omp parallel for schedule(static)
  for (int64_t n = 0; n < S->N; ++n) preprocess_one(S, n, cam, set, &pre[n]);
  return pre;
}

/* Which pixels to process: all (pix == NULL) or a list of flat indices. */
typedef struct {
  const scene_t* S;
  const double* cam;
  const double* set;
  const pre_t* pre;
  tiles_t tiles;
  int* all;        /* brute force candidate list 0..N-1 */
  int mode;        /* 0 brute force, 1 binned */
  int W, H, tx;
  int maxlist;
} ctx_t;

static void ctx_init(ctx_t* C, const scene_t* S, const double* cam, const double* set, int mode) {
  memset(C, 0, sizeof *C);
  C->S = S; C->cam = cam; C->set = set; C->mode = mode;
  C->W = (int)cam[CAM_W]; C->H = (int)cam[CAM_H];
  const int tile = (int)set[SET_TILE];
  C->tx = (C->W + tile - 1) / tile;
  const int ty = (C->H + tile - 1) / tile;
  C->pre = run_preprocess(S, cam, set);
  if (mode == 0) {
    C->all = (int*)malloc(sizeof(int) * (size_t)(S->N > 0 ? S->N : 1));
    for (int64_t n = 0; n < S->N; ++n) C->all[n] = (int)n;
    C->maxlist = (int)S->N;
  } else {
    C->tiles.tile = tile;
    build_tiles(C->pre, S->N, C->tx, ty, &C->tiles);
    int64_t mx = 0;
    for (int t = 0; t < C->tiles.ntiles; ++t) {
      const int64_t l = C->tiles.start[t + 1] - C->tiles.start[t];
      if (l > mx) mx = l;
    }
    C->maxlist = (int)mx;
  }
  if (C->maxlist < 1) C->maxlist = 1;
}
static void ctx_free(ctx_t* C) {
  free((void*)C->pre);
  free(C->all);
  free(C->tiles.start);
  free(C->tiles.idx);
}
static void pixel_list(const ctx_t* C, int i, int j, const int** cand, int* ncand) {
  if (C->mode == 0) { *cand = C->all; *ncand = (int)C->S->N; return; }
  const int tile = (int)C->set[SET_TILE];
  const int t = (j / tile) * C->tx + (i / tile);
  *cand = C->tiles.idx + C->tiles.start[t];
  *ncand = (int)(C->tiles.start[t + 1] - C->tiles.start[t]);
}

/* Render: out[12][H][W] (double), count[H][W], flags[H][W], dexact[H][W].
 * pix: optional list of flat pixel indices (npix of them); then the outputs
 * are written compactly, out[12][npix] etc.  shift (optional, [N][2]) moves
 * each surfel's opacity footprint on screen (for finite differences of the
 * screen-space densification gradient). */
int oracle_render(int64_t N, int deg, const double* mu, const double* quat, const double* scale,
                  const double* opac, const double* sh, const double* cam, const double* set,
                  int mode, int64_t npix, const int64_t* pix, const double* shift, double* out,
                  int* count, int* flags, double* dexact, int* ncand) {
  scene_t S = mk_scene(N, deg, mu, quat, scale, opac, sh);
  ctx_t C;
  ctx_init(&C, &S, cam, set, mode);
  const int64_t HW = (int64_t)C.W * C.H;
  const int64_t P = pix ? npix : HW;
#pragma omp parallel
  {
    pair_t* tmp = (pair_t*)malloc(sizeof(pair_t) * (size_t)C.maxlist);
    pair_t* bl = (pair_t*)malloc(sizeof(pair_t) * (size_t)C.maxlist);
    okey_t* keys = (okey_t*)malloc(sizeof(okey_t) * (size_t)C.maxlist);
#pragma omp for schedule(dynamic, 64)
    for (int64_t k = 0; k < P; ++k) {
      const int64_t f = pix ? pix[k] : k;
      const int i = (int)(f % C.W), j = (int)(f / C.W);
      const int* cand; int nc;
      pixel_list(&C, i, j, &cand, &nc);
      pix_t px;
      composite_pixel(C.pre, cand, nc, i + 0.5, j + 0.5, set, shift, tmp, keys, bl, &px);
      for (int c = 0; c < OUT_PLANES; ++c) out[c * P + k] = px.out[c];
      if (count) count[k] = px.count;
      if (dexact) dexact[k] = px.dexact;
      if (ncand) ncand[k] = px.ncand;
      if (flags) flags[k] = px.flags;
    }
    free(tmp); free(bl); free(keys);
  }
  ctx_free(&C);
  return 0;
}

/* Largest Jacobian condition number among the pairs blended at each pixel
 * (used by tests to separate ill-conditioned pixels). */
int oracle_pixel_cond(int64_t N, int deg, const double* mu, const double* quat, const double* scale,
                      const double* opac, const double* sh, const double* cam, const double* set,
                      double* maxcond) {
  scene_t S = mk_scene(N, deg, mu, quat, scale, opac, sh);
  ctx_t C;
  ctx_init(&C, &S, cam, set, 1);
  const int64_t HW = (int64_t)C.W * C.H;
#pragma omp parallel
  {
    pair_t* tmp = (pair_t*)malloc(sizeof(pair_t) * (size_t)C.maxlist);
    pair_t* bl = (pair_t*)malloc(sizeof(pair_t) * (size_t)C.maxlist);
    okey_t* keys = (okey_t*)malloc(sizeof(okey_t) * (size_t)C.maxlist);
#pragma omp for schedule(dynamic, 64)
    for (int64_t k = 0; k < HW; ++k) {
      const int i = (int)(k % C.W), j = (int)(k / C.W);
      const int* cand; int nc;
      pixel_list(&C, i, j, &cand, &nc);
      pix_t px;
      composite_pixel(C.pre, cand, nc, i + 0.5, j + 0.5, set, NULL, tmp, keys, bl, &px);
      double mc = 0;
      for (int b = 0; b < px.count; ++b)
        if (bl[b].obj && C.pre[bl[b].n].cond > mc) mc = C.pre[bl[b].n].cond;
      maxcond[k] = mc;
    }
    free(tmp); free(bl); free(keys);
  }
  ctx_free(&C);
  return 0;
}

/* ---------------------------------------------------------------------- */
/* Backward.                                                               */

static void atomic_add(double* p, double v) {
#pragma omp atomic
  *p += v;
}

/* Per-surfel intermediate gradient record, in the oracle's own variables. */
enum { G_M = 0 /* 9 */, G_RGB = 9 /* 3 */, G_OP = 12, G_N = 13 /* 3 */, G_LEN = 16 };

/* adj: n_sets x [11][H][W] adjoint planes (d loss / d output plane).
 * Set 0 drives parameter gradients; every set yields the screen-space
 * translation gradient (definition step 14) into sgrad[set][N][2].
 * Outputs: dmu[N*3], dq[N*4], ds[N*2], dop[N], dsh[N*K*3] (accumulated,
 * zero them first), sgrad (accumulated), gint[N*16] (intermediate record,
 * optional). */
int oracle_backward(int64_t N, int deg, const double* mu, const double* quat, const double* scale,
                    const double* opac, const double* sh, const double* cam, const double* set,
                    int n_sets, const double* adj, double* dmu, double* dq, double* ds, double* dop,
                    double* dsh, double* sgrad, double* gint) {
  scene_t S = mk_scene(N, deg, mu, quat, scale, opac, sh);
  ctx_t C;
  ctx_init(&C, &S, cam, set, 1);
  const int W = C.W, H = C.H;
  const int64_t HW = (int64_t)W * H;
  double* g = (double*)calloc((size_t)N * G_LEN, sizeof(double));
  const double sinv = set[SET_SCREEN_INV_S2];
#pragma omp parallel
  {
    pair_t* tmp = (pair_t*)malloc(sizeof(pair_t) * (size_t)C.maxlist);
    pair_t* bl = (pair_t*)malloc(sizeof(pair_t) * (size_t)C.maxlist);
    okey_t* keys = (okey_t*)malloc(sizeof(okey_t) * (size_t)C.maxlist);
    double* dLdw = (double*)malloc(sizeof(double) * (size_t)C.maxlist);
    double* suf = (double*)malloc(sizeof(double) * (size_t)(C.maxlist + 1));
    double* dLda = (double*)malloc(sizeof(double) * (size_t)C.maxlist);
#pragma omp for schedule(dynamic, 64)
    for (int64_t k = 0; k < HW; ++k) {
      const int i = (int)(k % W), j = (int)(k / W);
      const double x = i + 0.5, y = j + 0.5;
      const int* cand; int nc;
      pixel_list(&C, i, j, &cand, &nc);
      pix_t px;
      const int nb = composite_pixel(C.pre, cand, nc, x, y, set, NULL, tmp, keys, bl, &px);
      if (nb == 0) continue;
      const double Af = px.out[O_ALPHA], Zf = px.out[O_DEPTH], Tf = px.out[O_TFINAL];
      /* index of the median pair: last blended pair entered with T > 0.5 */
      int med = -1;
      for (int b = 0; b < nb; ++b) if (bl[b].T > 0.5) med = b;
      for (int s = 0; s < n_sets; ++s) {
        const double* a = adj + (size_t)s * ADJ_PLANES * HW;
        double gC[3], gN[3];
        for (int c = 0; c < 3; ++c) { gC[c] = a[(O_R + c) * HW + k]; gN[c] = a[(O_NX + c) * HW + k]; }
        const double gA = a[O_ALPHA * HW + k], gZ = a[O_DEPTH * HW + k];
        const double gI = a[O_INVDEPTH * HW + k], gMed = a[O_MEDIAN * HW + k];
        const double gD = a[O_DIST * HW + k];
        /* dL/dw_k for every blended pair, with the distortion sum written out
         * through prefix (A_{k-1}, Z_{k-1}) and suffix sums */
        double Ap = 0, Zp = 0;
        for (int b = 0; b < nb; ++b) {
          const pre_t* P = &C.pre[bl[b].n];
          const double z = bl[b].z;
          const double Ak = Ap + bl[b].w, Zk = Zp + bl[b].w * z;
          const double dD = 2.0 * (z * Ap - Zp + (Zf - Zk) - z * (Af - Ak));
          dLdw[b] = gC[0] * P->rgb[0] + gC[1] * P->rgb[1] + gC[2] * P->rgb[2] + gA + gZ * z +
                    gI / z + gN[0] * P->nrm[0] + gN[1] * P->nrm[1] + gN[2] * P->nrm[2] + gD * dD;
          Ap = Ak; Zp = Zk;
        }
        const double dLdTf = gC[0] * set[SET_BG] + gC[1] * set[SET_BG + 1] + gC[2] * set[SET_BG + 2];
        suf[nb] = Tf * dLdTf;
        for (int b = nb - 1; b >= 0; --b) suf[b] = suf[b + 1] + bl[b].w * dLdw[b];
        for (int b = 0; b < nb; ++b)
          dLda[b] = bl[b].T * dLdw[b] - suf[b + 1] / (1.0 - bl[b].alpha);
        Ap = 0;
        for (int b = 0; b < nb; ++b) {
          const pair_t* pr = &bl[b];
          const pre_t* P = &C.pre[pr->n];
          const double* M = P->M;
          const double z = pr->z;
          const double Ak = Ap + pr->w;
          /* alpha -> rho */
          const int unclamped = pr->araw < set[SET_ALPHA_MAX];
          const double dadrho = unclamped ? -0.5 * P->opac * pr->G : 0.0;
          const double dLdrho = dLda[b] * dadrho;
          /* d rho / d pixel position */
          double drx, dry;
          const double ccx = M[2] / M[8], ccy = M[5] / M[8];
          if (pr->obj) {
            const double gh[3] = {2 * pr->u / pr->h[2], 2 * pr->v / pr->h[2],
                                  -2 * (pr->u * pr->u + pr->v * pr->v) / pr->h[2]};
            double t1[3], t2[3];
            cross3(pr->l2, gh, t1);
            cross3(gh, pr->l1, t2);
            const double m3[3] = {M[6], M[7], M[8]};
            drx = -dot3(t1, m3);
            dry = -dot3(t2, m3);
          } else {
            drx = 2 * sinv * (x - ccx);
            dry = 2 * sinv * (y - ccy);
          }
          /* screen translation gradient: footprint moved by delta, so the
           * pixel sample moves by -delta relative to it */
          atomic_add(&sgrad[((size_t)s * N + pr->n) * 2 + 0], -dLdrho * drx);
          atomic_add(&sgrad[((size_t)s * N + pr->n) * 2 + 1], -dLdrho * dry);
          if (s != 0) { Ap = Ak; continue; }
          double* gn = g + (size_t)pr->n * G_LEN;
          for (int c = 0; c < 3; ++c) {
            atomic_add(&gn[G_RGB + c], pr->w * gC[c]);
            atomic_add(&gn[G_N + c], pr->w * gN[c]);
          }
          if (unclamped) atomic_add(&gn[G_OP], dLda[b] * pr->G);
          /* d L / d z for this pair */
          const double dDdz = 2.0 * pr->w * ((Ak - pr->w) - (Af - Ak));
          double dLdz = pr->w * (gZ - gI / (z * z)) + gD * dDdz + (b == med ? gMed : 0.0);
          double gM[9] = {0};
          if (pr->obj) {
            /* rho = u^2 + v^2; z = m3 . (u, v, 1) */
            const double dLdu = dLdrho * 2 * pr->u + dLdz * M[6];
            const double dLdv = dLdrho * 2 * pr->v + dLdz * M[7];
            gM[6] += dLdz * pr->u; gM[7] += dLdz * pr->v; gM[8] += dLdz;
            const double h3 = pr->h[2];
            const double gh[3] = {dLdu / h3, dLdv / h3, -(dLdu * pr->u + dLdv * pr->v) / h3};
            double gl1[3], gl2[3];
            cross3(pr->l2, gh, gl1);
            cross3(gh, pr->l1, gl2);
            for (int c = 0; c < 3; ++c) {
              gM[c] += gl1[c];
              gM[3 + c] += gl2[c];
              gM[6 + c] += -x * gl1[c] - y * gl2[c];
            }
          } else {
            /* rho = sinv |x - c|^2, c = (M13/M33, M23/M33); z = M33 */
            const double dcx = dLdrho * 2 * sinv * (ccx - x);
            const double dcy = dLdrho * 2 * sinv * (ccy - y);
            gM[2] += dcx / M[8];
            gM[5] += dcy / M[8];
            gM[8] += -(dcx * ccx + dcy * ccy) / M[8] + dLdz;
          }
          for (int c = 0; c < 9; ++c) if (gM[c] != 0) atomic_add(&gn[G_M + c], gM[c]);
          Ap = Ak;
        }
      }
    }
    free(tmp); free(bl); free(keys); free(dLdw); free(suf); free(dLda);
  }
  /* chain the per-surfel record to the parameters */
  const double* Rc = cam + CAM_R;
  const double fx = cam[CAM_FX], fy = cam[CAM_FY], cx = cam[CAM_CX], cy = cam[CAM_CY];
  double o[3];
  cam_pos(cam, o);
#pragma omp parallel for schedule(static)
  for (int64_t n = 0; n < N; ++n) {
    const pre_t* P = &C.pre[n];
    if (!P->live) continue;
    const double* gn = g + (size_t)n * G_LEN;
    if (gint) memcpy(gint + (size_t)n * G_LEN, gn, sizeof(double) * G_LEN);
    double q[4] = {S.quat[4 * n], S.quat[4 * n + 1], S.quat[4 * n + 2], S.quat[4 * n + 3]};
    const double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int c = 0; c < 4; ++c) q[c] /= qn;
    double R[9];
    quat_to_R(q, R);
    const double r1[3] = {R[0], R[3], R[6]}, r2[3] = {R[1], R[4], R[7]}, r3[3] = {R[2], R[5], R[8]};
    const double mu_[3] = {S.mu[3 * n], S.mu[3 * n + 1], S.mu[3 * n + 2]};
    const double su = S.scale[2 * n], sv = S.scale[2 * n + 1];
    double p[3], tu[3], tv[3], nv[3];
    matvec3(Rc, mu_, p);
    for (int c = 0; c < 3; ++c) p[c] += cam[CAM_T + c];
    matvec3(Rc, r1, tu);
    matvec3(Rc, r2, tv);
    matvec3(Rc, r3, nv);
    /* M = K B, B = [a | b | p]:  dB = K^T dM */
    const double* gM = gn + G_M;
    double dB[9];
    /* K = [[fx,0,cx],[0,fy,cy],[0,0,1]]; (K^T G)_{rc} = sum_i K_{ir} G_{ic} */
    for (int c = 0; c < 3; ++c) {
      dB[0 * 3 + c] = fx * gM[0 * 3 + c];
      dB[1 * 3 + c] = fy * gM[1 * 3 + c];
      dB[2 * 3 + c] = cx * gM[0 * 3 + c] + cy * gM[1 * 3 + c] + gM[2 * 3 + c];
    }
    const double da[3] = {dB[0], dB[3], dB[6]}, db[3] = {dB[1], dB[4], dB[7]};
    const double dp[3] = {dB[2], dB[5], dB[8]};
    ds[2 * n] += dot3(da, tu);
    ds[2 * n + 1] += dot3(db, tv);
    double dr1[3], dr2[3], dr3[3], dmuv[3];
    matTvec3(Rc, da, dr1);
    matTvec3(Rc, db, dr2);
    for (int c = 0; c < 3; ++c) { dr1[c] *= su; dr2[c] *= sv; }
    const double sgn = dot3(nv, p) > 0 ? -1.0 : 1.0;
    const double dnv[3] = {sgn * gn[G_N], sgn * gn[G_N + 1], sgn * gn[G_N + 2]};
    matTvec3(Rc, dnv, dr3);
    matTvec3(Rc, dp, dmuv);
    /* colour: rgb = max(0, sum sh Y(dir) + 0.5), dir = (mu - o)/|mu - o| */
    double d[3];
    for (int c = 0; c < 3; ++c) d[c] = mu_[c] - o[c];
    const double dl = sqrt(dot3(d, d));
    for (int c = 0; c < 3; ++c) d[c] /= dl;
    double Y[16], dY[16][3];
    sh_basis(d, Y, dY);
    double ddir[3] = {0, 0, 0};
    for (int c = 0; c < 3; ++c) {
      if (!(P->rawcol[c] > 0)) continue;
      const double gc = gn[G_RGB + c];
      for (int kk = 0; kk < S.K; ++kk) {
        dsh[(n * S.K + kk) * 3 + c] += gc * Y[kk];
        const double f = S.sh[(n * S.K + kk) * 3 + c];
        for (int e = 0; e < 3; ++e) ddir[e] += gc * f * dY[kk][e];
      }
    }
    const double dd = dot3(d, ddir);
    for (int c = 0; c < 3; ++c) dmuv[c] += (ddir[c] - d[c] * dd) / dl;
    for (int c = 0; c < 3; ++c) dmu[3 * n + c] += dmuv[c];
    /* rotation: columns r1, r2, r3 of R(q_hat) */
    double GR[9];
    for (int rr = 0; rr < 3; ++rr) { GR[3 * rr] = dr1[rr]; GR[3 * rr + 1] = dr2[rr]; GR[3 * rr + 2] = dr3[rr]; }
    double dqh[4];
    quat_to_R_vjp(q, GR, dqh);
    const double qd = q[0] * dqh[0] + q[1] * dqh[1] + q[2] * dqh[2] + q[3] * dqh[3];
    for (int c = 0; c < 4; ++c) dq[4 * n + c] += (dqh[c] - q[c] * qd) / qn;
    dop[n] += gn[G_OP];
  }
  free(g);
  ctx_free(&C);
  return 0;
}

/* ---------------------------------------------------------------------- */
/* Losses (Sec. 3.1: L1 + D-SSIM; Sec. 3.2: depth loss on inverse depth).    */

/* 11x11 Gaussian window, sigma 1.5, normalised to unit sum. */
static void gauss_window(double w[11]) {
  double s = 0;
  for (int i = 0; i < 11; ++i) { w[i] = exp(-((i - 5) * (i - 5)) / (2 * 1.5 * 1.5)); s += w[i]; }
  for (int i = 0; i < 11; ++i) w[i] /= s;
}

/* Windowed mean of f at every pixel, zero padded ("same"), written as the
 * direct 2-D double sum over the 11x11 window. */
static void window_sum(const double* f, int W, int H, double* o) {
  double g[11];
  gauss_window(g);
#pragma omp parallel for schedule(static)
  for (int j = 0; j < H; ++j)
    for (int i = 0; i < W; ++i) {
      double acc = 0;
      for (int b = -5; b <= 5; ++b) {
        const int jj = j + b;
        if (jj < 0 || jj >= H) continue;
        for (int a = -5; a <= 5; ++a) {
          const int ii = i + a;
          if (ii < 0 || ii >= W) continue;
          acc += g[a + 5] * g[b + 5] * f[(int64_t)jj * W + ii];
        }
      }
      o[(int64_t)j * W + i] = acc;
    }
}

/* SSIM of two single-channel images and its gradient w.r.t. x.
 * Returns the sum over pixels of the SSIM map; dssim (optional) receives
 * d(sum map)/dx. */
static double ssim_channel(const double* X, const double* Yt, int W, int H, double* dssim) {
  const int64_t n = (int64_t)W * H;
  const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
  double* buf = (double*)malloc(sizeof(double) * (size_t)n * 10);
  double *xx = buf, *yy = buf + n, *xy = buf + 2 * n;
  double *mx = buf + 3 * n, *my = buf + 4 * n, *sxx = buf + 5 * n, *syy = buf + 6 * n, *sxy = buf + 7 * n;
  for (int64_t k = 0; k < n; ++k) { xx[k] = X[k] * X[k]; yy[k] = Yt[k] * Yt[k]; xy[k] = X[k] * Yt[k]; }
  window_sum(X, W, H, mx);
  window_sum(Yt, W, H, my);
  window_sum(xx, W, H, sxx);
  window_sum(yy, W, H, syy);
  window_sum(xy, W, H, sxy);
  double total = 0;
  double *gmx = xx, *gsxx = yy, *gsxy = xy; /* reuse as partials */
  for (int64_t k = 0; k < n; ++k) {
    const double ux = mx[k], uy = my[k];
    const double vx = sxx[k] - ux * ux, vy = syy[k] - uy * uy, cxy = sxy[k] - ux * uy;
    const double A1 = 2 * ux * uy + C1, A2 = 2 * cxy + C2;
    const double B1 = ux * ux + uy * uy + C1, B2 = vx + vy + C2;
    const double s = (A1 * A2) / (B1 * B2);
    total += s;
    /* partials of s w.r.t. the windowed moments mu_x, E[x^2], E[xy] */
    const double ds_dux_direct = (2 * uy * A2) / (B1 * B2) - s * (2 * ux) / B1;
    const double ds_dvx = -s / B2;        /* d s / d var_x */
    const double ds_dcxy = 2 * A1 / (B1 * B2);
    /* var_x = E[x^2] - ux^2, cov = E[xy] - ux uy */
    gmx[k] = ds_dux_direct + ds_dvx * (-2 * ux) + ds_dcxy * (-uy);
    gsxx[k] = ds_dvx;
    gsxy[k] = ds_dcxy;
  }
  if (dssim) {
    double* t1 = buf + 8 * n;
    double* t2 = buf + 9 * n;
    /* the window is symmetric, so the adjoint of the windowed sum is the
     * same windowed sum */
    window_sum(gmx, W, H, t1);
    for (int64_t k = 0; k < n; ++k) dssim[k] = t1[k];
    window_sum(gsxx, W, H, t1);
    window_sum(gsxy, W, H, t2);
    for (int64_t k = 0; k < n; ++k) dssim[k] += 2 * X[k] * t1[k] + Yt[k] * t2[k];
  }
  free(buf);
  return total;
}

/* out: rendered planes [12][H][W]; tgt: [3][H][W]; tinv: [H][W] (may be NULL).
 * w: [w_l1, w_ssim, w_depth].  losses: [L1, SSIM, Ldepth, total].
 * adj_total/adj_ssim/adj_l1: [11][H][W] adjoint planes (zeroed here). */
int oracle_loss(int W, int H, const double* out, const double* tgt, const double* tinv,
                const double* w, double* losses, double* adj_total, double* adj_ssim,
                double* adj_l1) {
  const int64_t n = (int64_t)W * H;
  memset(adj_total, 0, sizeof(double) * (size_t)ADJ_PLANES * n);
  memset(adj_ssim, 0, sizeof(double) * (size_t)ADJ_PLANES * n);
  memset(adj_l1, 0, sizeof(double) * (size_t)ADJ_PLANES * n);
  double l1 = 0, ss = 0, ld = 0;
  double* ds = (double*)malloc(sizeof(double) * (size_t)n);
  for (int c = 0; c < 3; ++c) {
    const double* X = out + (O_R + c) * n;
    const double* T = tgt + c * n;
    for (int64_t k = 0; k < n; ++k) {
      const double d = X[k] - T[k];
      l1 += fabs(d);
      const double sg = d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0);
      adj_l1[(O_R + c) * n + k] = w[0] * sg / (3.0 * n);
    }
    ss += ssim_channel(X, T, W, H, ds);
    for (int64_t k = 0; k < n; ++k) adj_ssim[(O_R + c) * n + k] = -w[1] * ds[k] / (3.0 * n);
  }
  free(ds);
  l1 /= 3.0 * n;
  ss /= 3.0 * n;
  if (tinv) {
    for (int64_t k = 0; k < n; ++k) {
      const double d = out[O_INVDEPTH * n + k] - tinv[k];
      ld += fabs(d);
      const double sg = d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0);
      adj_total[O_INVDEPTH * n + k] = w[2] * sg / (double)n;
    }
    ld /= (double)n;
  }
  for (int c = 0; c < 3; ++c)
    for (int64_t k = 0; k < n; ++k)
      adj_total[(O_R + c) * n + k] = adj_l1[(O_R + c) * n + k] + adj_ssim[(O_R + c) * n + k];
  losses[0] = l1;
  losses[1] = ss;
  losses[2] = ld;
  losses[3] = w[0] * l1 + w[1] * (1.0 - ss) + w[2] * ld;
  return 0;
}

/* SSIM of single-channel images (sum of the map) and its gradient, exported
 * for the pins. */
double oracle_ssim_sum(int W, int H, const double* X, const double* Y, double* grad) {
  return ssim_channel(X, Y, W, H, grad);
}

/* ---------------------------------------------------------------------- */
/* Densification statistics and selection (Sec. 3.1, Sec. 3.2 Eq. 2, eta).  */

/* stats[N][4] = S_tot, S_ssim, S_l1, cnt; sgrad[3][N][2]; live[N] visible. */
int oracle_densify_accumulate(int64_t N, const double* sgrad, const int* visible, double* stats) {
  for (int64_t n = 0; n < N; ++n) {
    if (!visible[n]) continue;
    for (int s = 0; s < 3; ++s) {
      const double gx = sgrad[((size_t)s * N + n) * 2], gy = sgrad[((size_t)s * N + n) * 2 + 1];
      stats[4 * n + s] += sqrt(gx * gx + gy * gy);
    }
    stats[4 * n + 3] += 1.0;
  }
  return 0;
}

/* Eq. 2: scale = max(omega * avg|grad L| / avg|grad L_SSIM|, 1); g = scale *
 * S_ssim/cnt; eligible = g >= grad_thr and eta >= eta_thr and cnt > 0.
 * Averages are over surfels with cnt > 0 of the per-surfel view means. */
int oracle_densify_select(int64_t N, const double* stats, const double* scale, double omega,
                          double grad_thr, double eta_thr, unsigned char* mask, double* g_out,
                          double* scale_out) {
  double st = 0, ss = 0;
  int64_t m = 0;
  for (int64_t n = 0; n < N; ++n) {
    const double c = stats[4 * n + 3];
    if (c > 0) { st += stats[4 * n] / c; ss += stats[4 * n + 1] / c; ++m; }
  }
  double k = 1.0;
  if (m > 0 && ss > 0) {
    const double r = omega * (st / m) / (ss / m);
    k = r > 1.0 ? r : 1.0;
  }
  if (scale_out) *scale_out = k;
  for (int64_t n = 0; n < N; ++n) {
    const double c = stats[4 * n + 3];
    const double gg = c > 0 ? k * stats[4 * n + 1] / c : 0.0;
    const double su = scale[2 * n], sv = scale[2 * n + 1];
    const double eta = fmin(su, sv) / fmax(su, sv);
    g_out[n] = gg;
    mask[n] = (unsigned char)(c > 0 && gg >= grad_thr && eta >= eta_thr);
  }
  return 0;
}

/* Elongation filter: keep[n] = eta_n >= eta_thr, eta = min(s)/max(s). */
int oracle_elongation(int64_t N, const double* scale, double eta_thr, unsigned char* keep) {
  for (int64_t n = 0; n < N; ++n) {
    const double su = scale[2 * n], sv = scale[2 * n + 1];
    keep[n] = (unsigned char)(fmin(su, sv) / fmax(su, sv) >= eta_thr);
  }
  return 0;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Tile lists of the binned mode in compositing order: start[ntiles + 1]
 * offsets, idx[K] surfel indices (sorted per tile by FP32 centre depth,
 * then index). */
int oracle_tile_lists(int64_t N, int deg, const double* mu, const double* quat, const double* scale,
                      const double* opac, const double* sh, const double* cam, const double* set,
                      int64_t* start, int* idx) {
  scene_t S = mk_scene(N, deg, mu, quat, scale, opac, sh);
  ctx_t C;
  ctx_init(&C, &S, cam, set, 1);
  memcpy(start, C.tiles.start, sizeof(int64_t) * (size_t)(C.tiles.ntiles + 1));
  const int64_t K = C.tiles.start[C.tiles.ntiles];
  memcpy(idx, C.tiles.idx, sizeof(int) * (size_t)K);
#pragma omp parallel for schedule(dynamic, 16)
  for (int t = 0; t < C.tiles.ntiles; ++t) {
    const int64_t a = start[t], b = start[t + 1];
    okey_t* k = (okey_t*)malloc(sizeof(okey_t) * (size_t)(b - a + 1));
    for (int64_t i = a; i < b; ++i) { k[i - a].z = C.pre[idx[i]].zkey; k[i - a].n = idx[i]; k[i - a].slot = 0; }
    qsort(k, (size_t)(b - a), sizeof(okey_t), cmp_keys);
    for (int64_t i = a; i < b; ++i) idx[i] = k[i - a].n;
    free(k);
  }
  ctx_free(&C);
  return 0;
}

/* ---------------------------------------------------------------------- */
/* Trim contribution (Sec. 3.3, Eq. 3).                                     */

/* Single-view contribution of every surfel, as its two parts: for surfel n,
 *   count[n] = |P_k|, the pixels of the view inside n's projected region
 *              (its 3-sigma support rho <= rho_max, occluded or not), and
 *   sum[n]   = sum over those pixels of alpha^gamma * T^(1 - gamma), with
 *              alpha the opacity the compositing applied to the pair (0 for a
 *              pair below the alpha cutoff or behind the pixel's stop) and T
 *              the transmittance in front of n on that pixel (the product of
 *              (1 - alpha_j) over the pairs composited before it),
 * so that C_{n,k} = sum[n] / count[n] (0 when count[n] = 0).
 * Decisions within a hair of a threshold, where an FP32 implementation may
 * legitimately decide the other way, are reported per surfel:
 *   flag_count[n]: pixels where n's own rho is within 1e-4 of rho_max (its
 *                  membership in P_k is uncertain);
 *   flag_sum[n]:   pixels of n's (near-)support where some decision at or in
 *                  front of n was near its threshold (rho near rho_max, alpha
 *                  near the cutoff, the stop near T_min), so that n's alpha or
 *                  T there is uncertain.
 * Outputs are overwritten. */
int oracle_contribution(int64_t N, int deg, const double* mu, const double* quat, const double* scale,
                        const double* opac, const double* sh, const double* cam, const double* set,
                        int mode, double gamma, double* sum, int64_t* count, int64_t* flag_count,
                        int64_t* flag_sum) {
  scene_t S = mk_scene(N, deg, mu, quat, scale, opac, sh);
  ctx_t C;
  ctx_init(&C, &S, cam, set, mode);
  for (int64_t n = 0; n < N; ++n) { sum[n] = 0.0; count[n] = 0; flag_count[n] = 0; flag_sum[n] = 0; }
  const int64_t HW = (int64_t)C.W * C.H;
  const double rmax = set[SET_RHO_MAX];
#pragma omp parallel
  {
    pair_t* sup = (pair_t*)malloc(sizeof(pair_t) * (size_t)C.maxlist);
    okey_t* keys = (okey_t*)malloc(sizeof(okey_t) * (size_t)C.maxlist);
#pragma omp for schedule(dynamic, 64)
    for (int64_t f = 0; f < HW; ++f) {
      const int i = (int)(f % C.W), j = (int)(f / C.W);
      const double x = i + 0.5, y = j + 0.5;
      const int* cand; int nc;
      pixel_list(&C, i, j, &cand, &nc);
      /* the pixel's support pairs and those within the margin outside it,
       * in compositing order */
      int m = 0;
      for (int c = 0; c < nc; ++c) {
        const int n = cand[c];
        if (!C.pre[n].live) continue;
        pair_t pr;
        eval_pair(&C.pre[n], n, x, y, set, &pr);
        if (!(pr.rho <= rmax + 1e-4)) continue;
        sup[m] = pr;
        keys[m].z = C.pre[n].zkey; keys[m].n = n; keys[m].slot = m;
        ++m;
      }
      qsort(keys, (size_t)m, sizeof(okey_t), cmp_keys);
      double T = 1.0;
      int stopped = 0, taint = 0;
      for (int k = 0; k < m; ++k) {
        const pair_t* pr = &sup[keys[k].slot];
        const int n = keys[k].n;
        const int in = pr->rho <= rmax;
        if (fabs(pr->rho - rmax) < 1e-4) {
          taint = 1;
#pragma omp atomic
          flag_count[n] += 1;
        }
        double a = 0.0;  /* opacity the compositing applies */
        if (in) {
          if (fabs(pr->alpha / set[SET_ALPHA_MIN] - 1.0) < 1e-5) taint = 1;
          if (!stopped && pr->alpha >= set[SET_ALPHA_MIN]) {
            const double Tn = T * (1.0 - pr->alpha);
            if (fabs(Tn / set[SET_T_MIN] - 1.0) < 1e-5) taint = 1;
            if (Tn < set[SET_T_MIN]) stopped = 1;
            else a = pr->alpha;
          }
        }
        if (taint) {
#pragma omp atomic
          flag_sum[n] += 1;
        }
        if (!in) continue;
#pragma omp atomic
        count[n] += 1;
        if (a > 0.0) {
          atomic_add(&sum[n], pow(a, gamma) * pow(T, 1.0 - gamma));
          T *= 1.0 - a;
        }
      }
    }
    free(sup); free(keys);
  }
  ctx_free(&C);
  return 0;
}

/* ---------------------------------------------------------------------- */
/* Visible frequency of points (Sec. 4, crop volume estimation).         */

/* Each point is an isotropic 3D Gaussian of standard deviation sigma.  In a
 * view (camera array as above) it is visible when it lies in front of the
 * near plane and the 3-sigma square of its projected footprint overlaps the
 * image: the footprint's covariance is the EWA projection sigma^2 J J^T of the
 * isotropic covariance (J the Jacobian of the perspective projection at the
 * point) plus the rasterizer's low-pass of lowpass px^2 on both axes, its
 * 3-sigma half-width r = 3 sqrt(largest eigenvalue), and the square
 * [c - r, c + r]^2 around the projected centre c must meet [0, W] x [0, H]
 * with positive overlap.  count[j] += the number of visible views;
 * flagged[j] += the views where a decision was within 2e-6 (relative to the
 * magnitudes involved) of its threshold, beyond what an FP32 evaluation can
 * resolve. */
int oracle_visibility_count(int64_t N, const double* pts, double sigma, int V, const double* cams,
                            double near, double lowpass, int64_t* count, int64_t* flagged) {
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < N; ++j) {
    int64_t c = 0, f = 0;
    for (int v = 0; v < V; ++v) {
      const double* cm = cams + (size_t)v * CAM_LEN;
      double p[3];
      matvec3(cm + CAM_R, pts + 3 * j, p);
      for (int i = 0; i < 3; ++i) p[i] += cm[CAM_T + i];
      const double z = p[2];
      if (fabs(z - near) <= 2e-6 * (fabs(z) + fabs(near))) ++f;
      if (!(z > near)) continue;
      const double fx = cm[CAM_FX], fy = cm[CAM_FY];
      /* J = [[fx/z, 0, -fx x/z^2], [0, fy/z, -fy y/z^2]] */
      const double J[2][3] = {{fx / z, 0.0, -fx * p[0] / (z * z)}, {0.0, fy / z, -fy * p[1] / (z * z)}};
      double S[2][2];
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
          S[a][b] = sigma * sigma * (J[a][0] * J[b][0] + J[a][1] * J[b][1] + J[a][2] * J[b][2]) +
                    (a == b ? lowpass : 0.0);
      const double mid = 0.5 * (S[0][0] + S[1][1]);
      const double half = 0.5 * (S[0][0] - S[1][1]);
      const double lmax = mid + sqrt(half * half + S[0][1] * S[0][1]);
      const double r = 3.0 * sqrt(lmax);
      const double cx = fx * p[0] / z + cm[CAM_CX], cy = fy * p[1] / z + cm[CAM_CY];
      const double W = cm[CAM_W], H = cm[CAM_H];
      const double m[4] = {cx + r, W - (cx - r), cy + r, H - (cy - r)};  /* all > 0: overlap */
      int vis = 1;
      for (int k = 0; k < 4; ++k) {
        const double scale = fabs(cx) + fabs(cy) + r + W + H;
        if (fabs(m[k]) <= 2e-6 * scale) ++f;
        if (!(m[k] > 0.0)) vis = 0;
      }
      c += vis;
    }
    count[j] += c;
    flagged[j] += f;
  }
  return 0;
}
