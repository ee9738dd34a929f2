// FP64 CPU oracle for the FE-4DGS differentiable rasterization pass.
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
// cpu_baseline / reference legs of bench.py may load this library.  The
// product path never calls it; it shares no code, header, table or constant
// with the CUDA library.
//
// What it computes, by passage of arXiv 2503.06161 (FeatureEndo-4DGS):
//   * Gaussian density and covariance Sigma = R S S^T R^T (Sec. 3.1, Eq. 1-2).
//   * FST deformation: HexPlane sample -> MLP -> heads d_mu, d_R, d_S, d_o
//     (Sec. 3.2, Eq. 4; Appendix A) applied as G_t (Eq. 6).
//   * EWA projection Sigma' = J W Sigma W^T J^T (Sec. 3.3, Eq. 9 of the
//     rendering subsection).
//   * Front-to-back alpha blending of colour, semantic feature and depth in one
//     pass (Sec. 3.3, Eq. 7-8).
//   * The analytic reverse pass of all of the above (hand-derived, FP64).
//
// It is the plain definition: every pixel gathers its candidate Gaussians by
// scanning ALL Gaussians, sorts them by (depth, index), and runs the alpha/T
// recurrence.  There is no tiling.  Readings where the paper is silent
// (thresholds, dilation, SH basis, HexPlane combination) are listed in the
// project's design notes and restated at each use below.
//
// Build: g++ -O2 -std=c++17 -fopenmp -ffp-contract=off -shared -fPIC
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {

typedef struct {
  int P, D, sh_degree;
  const double *means;       // [P,3]
  const double *log_scales;  // [P,3]
  const double *quats;       // [P,4] (w,x,y,z), need not be unit length
  const double *logits;      // [P] opacity logits
  const double *sh;          // [P,16,3]
  const double *feat;        // [P,D] semantic feature z
} or_scene;

typedef struct {
  int enabled;        // 0: static scene (all offsets zero)
  int C, R;           // plane channels, plane resolution (R x R, all 6 planes)
  const double *planes;  // [6,R,R,C]: xy, xz, yz, xt, yt, zt; first index along
                         // the first coordinate of the pair, second along the second
  const double *w1, *b1;  // [64,C], [64]
  const double *w2, *b2;  // [64,64], [64]
  const double *wh, *bh;  // [11,64], [11]: d_mu(3) d_q(4) d_s(3) d_o(1)
  double bbox_min[3], bbox_max[3];
  const double *noise;    // [P,3] or NULL: d_mu += noise_scale * t * xi
  double noise_scale;
} or_deform;

typedef struct {
  int width, height;
  double fx, fy, cx, cy;
  double view[16];    // world->camera, row-major 4x4
  double campos[3];   // camera centre, world space
  double znear;
} or_camera;

// Per-Gaussian state after deformation and projection.
typedef struct {
  double *delta;     // [P,11]
  double *uv;        // [P,2] projected centre, pixel units
  double *conic;     // [P,3] inverse 2D covariance (a, b, c)
  double *opacity;   // [P]
  double *depth;     // [P] camera-space z of the centre
  double *rgb;       // [P,3] clamped at 0
  double *rgb_raw;   // [P,3]
  int *radius;       // [P] 0 = culled
  int *rect;         // [P,4] inclusive pixel rect x0,y0,x1,y1 (x0>x1: empty)
  double *rmargin;   // [P] distance of 3*sqrt(lambda) to the nearest integer, relative
  int *gflags;       // [P] bit0 rgb clamp, bit1 J clamp, bit2 relu, bit3 grid cell
  int *gndec;        // [P] number of near-threshold gradient-only decisions (may be NULL)
} or_gauss;

}  // extern "C"

namespace {

const double kPi = 3.14159265358979323846;
const int kHidden = 64;
const int kMaxC = 64;
const int kMaxD = 256;

// Thresholds of the compositing recurrence (readings; the paper gives none).
const double kAlphaMin = 1.0 / 255.0;
const double kAlphaMax = 0.99;
const double kTMin = 1e-4;
const double kDilation = 0.3;

// ---------------------------------------------------------------------------
// Real spherical harmonics, degree <= 3.
// Normalisation K_l^m = sqrt((2l+1)/(4 pi) * (l-m)!/(l+m)!), associated
// Legendre functions with the Condon-Shortley phase, real form
//   m<0: sqrt2 K P_l^|m| sin(|m| phi);  m=0: K P_l^0;  m>0: sqrt2 K P_l^m cos(m phi)
// written as polynomials in the unit direction (x,y,z); index l*l+l+m.
// ---------------------------------------------------------------------------
double fact(int n) { double r = 1; for (int i = 2; i <= n; ++i) r *= i; return r; }
double Klm(int l, int m) { return std::sqrt((2 * l + 1) / (4 * kPi) * fact(l - m) / fact(l + m)); }

struct ShConst {
  double c[16];
  ShConst() {
    const double s2 = std::sqrt(2.0);
    c[0] = Klm(0, 0);
    // l=1: P_1^0 = z, P_1^1 = -sin(theta)
    c[1] = -s2 * Klm(1, 1);  // * y
    c[2] = Klm(1, 0);        // * z
    c[3] = -s2 * Klm(1, 1);  // * x
    // l=2: P_2^0 = (3z^2-1)/2, P_2^1 = -3 z sin, P_2^2 = 3 sin^2
    c[4] = s2 * Klm(2, 2) * 3.0 * 2.0;  // * xy           (sin^2 sin2phi = 2xy)
    c[5] = -s2 * Klm(2, 1) * 3.0;       // * yz
    c[6] = Klm(2, 0) * 0.5;             // * (3z^2-1) = (2z^2-x^2-y^2)
    c[7] = -s2 * Klm(2, 1) * 3.0;       // * xz
    c[8] = s2 * Klm(2, 2) * 3.0;        // * (x^2-y^2)
    // l=3: P_3^0 = (5z^3-3z)/2, P_3^1 = -(3/2)(5z^2-1) sin,
    //      P_3^2 = 15 z sin^2, P_3^3 = -15 sin^3
    c[9] = -s2 * Klm(3, 3) * 15.0;        // * y(3x^2-y^2)
    c[10] = s2 * Klm(3, 2) * 15.0 * 2.0;  // * xyz
    c[11] = -s2 * Klm(3, 1) * 1.5;        // * y(4z^2-x^2-y^2)
    c[12] = Klm(3, 0) * 0.5;              // * z(2z^2-3x^2-3y^2)
    c[13] = -s2 * Klm(3, 1) * 1.5;        // * x(4z^2-x^2-y^2)
    c[14] = s2 * Klm(3, 2) * 15.0;        // * z(x^2-y^2)
    c[15] = -s2 * Klm(3, 3) * 15.0;       // * x(x^2-3y^2)
  }
};
const ShConst kSh;

// Basis values Y[16] and gradients dY[16][3] with respect to (x,y,z).
void sh_basis(const double d[3], double Y[16], double dY[16][3]) {
  const double x = d[0], y = d[1], z = d[2];
  const double* c = kSh.c;
  double poly[16], g[16][3];
  poly[0] = 1; g[0][0] = g[0][1] = g[0][2] = 0;
  poly[1] = y; g[1][0] = 0; g[1][1] = 1; g[1][2] = 0;
  poly[2] = z; g[2][0] = 0; g[2][1] = 0; g[2][2] = 1;
  poly[3] = x; g[3][0] = 1; g[3][1] = 0; g[3][2] = 0;
  poly[4] = x * y; g[4][0] = y; g[4][1] = x; g[4][2] = 0;
  poly[5] = y * z; g[5][0] = 0; g[5][1] = z; g[5][2] = y;
  poly[6] = 2 * z * z - x * x - y * y; g[6][0] = -2 * x; g[6][1] = -2 * y; g[6][2] = 4 * z;
  poly[7] = x * z; g[7][0] = z; g[7][1] = 0; g[7][2] = x;
  poly[8] = x * x - y * y; g[8][0] = 2 * x; g[8][1] = -2 * y; g[8][2] = 0;
  poly[9] = y * (3 * x * x - y * y); g[9][0] = 6 * x * y; g[9][1] = 3 * x * x - 3 * y * y; g[9][2] = 0;
  poly[10] = x * y * z; g[10][0] = y * z; g[10][1] = x * z; g[10][2] = x * y;
  poly[11] = y * (4 * z * z - x * x - y * y);
  g[11][0] = -2 * x * y; g[11][1] = 4 * z * z - x * x - 3 * y * y; g[11][2] = 8 * y * z;
  poly[12] = z * (2 * z * z - 3 * x * x - 3 * y * y);
  g[12][0] = -6 * x * z; g[12][1] = -6 * y * z; g[12][2] = 6 * z * z - 3 * x * x - 3 * y * y;
  poly[13] = x * (4 * z * z - x * x - y * y);
  g[13][0] = 4 * z * z - 3 * x * x - y * y; g[13][1] = -2 * x * y; g[13][2] = 8 * x * z;
  poly[14] = z * (x * x - y * y); g[14][0] = 2 * x * z; g[14][1] = -2 * y * z; g[14][2] = x * x - y * y;
  poly[15] = x * (x * x - 3 * y * y); g[15][0] = 3 * x * x - 3 * y * y; g[15][1] = -6 * x * y; g[15][2] = 0;
  for (int k = 0; k < 16; ++k) {
    Y[k] = c[k] * poly[k];
    for (int a = 0; a < 3; ++a) dY[k][a] = c[k] * g[k][a];
  }
}

// ---------------------------------------------------------------------------
// FST deformation (Sec. 3.2, Eq. 4-6; Appendix A), single-resolution reading:
// coordinates normalised to [-1,1] by the scene box (t in [0,1] -> [-1,1]);
// six planes xy,xz,yz,xt,yt,zt sampled bilinearly (grid corners at +-1,
// positions clamped to the border); f = elementwise product of the six
// samples; h1 = relu(W1 f + b1); h2 = relu(W2 h1 + b2); delta = Wh h2 + bh.
// ---------------------------------------------------------------------------
const int kPair[6][2] = {{0, 1}, {0, 2}, {1, 2}, {0, 3}, {1, 3}, {2, 3}};

struct DeformState {
  double coord[4];      // normalised coordinates in [-1,1] (unclamped)
  double pos[6][2];     // grid positions
  int clamped[6][2];
  int i0[6][2];
  double fr[6][2];
  double samp[6][kMaxC];
  double f[kMaxC];
  double pre1[kHidden], h1[kHidden], pre2[kHidden], h2[kHidden];
  double delta[11];
};

void deform_forward(const or_deform& df, const double mu[3], double t, DeformState& s) {
  const int C = df.C, R = df.R;
  for (int a = 0; a < 3; ++a)
    s.coord[a] = 2.0 * (mu[a] - df.bbox_min[a]) / (df.bbox_max[a] - df.bbox_min[a]) - 1.0;
  s.coord[3] = 2.0 * t - 1.0;
  for (int c = 0; c < C; ++c) s.f[c] = 1.0;
  for (int k = 0; k < 6; ++k) {
    for (int e = 0; e < 2; ++e) {
      double g = (s.coord[kPair[k][e]] + 1.0) * 0.5 * (R - 1);
      s.clamped[k][e] = 0;
      if (g < 0) { g = 0; s.clamped[k][e] = 1; }
      if (g > R - 1) { g = R - 1; s.clamped[k][e] = 1; }
      int i = (int)std::floor(g);
      if (i > R - 2) i = R - 2;
      s.pos[k][e] = g;
      s.i0[k][e] = i;
      s.fr[k][e] = g - i;
    }
    const double f1 = s.fr[k][0], f2 = s.fr[k][1];
    const int i = s.i0[k][0], j = s.i0[k][1];
    const double* P00 = df.planes + ((size_t)(k * R + i) * R + j) * C;
    const double* P10 = df.planes + ((size_t)(k * R + i + 1) * R + j) * C;
    const double* P01 = df.planes + ((size_t)(k * R + i) * R + j + 1) * C;
    const double* P11 = df.planes + ((size_t)(k * R + i + 1) * R + j + 1) * C;
    for (int c = 0; c < C; ++c) {
      double v = (1 - f1) * (1 - f2) * P00[c] + f1 * (1 - f2) * P10[c] + (1 - f1) * f2 * P01[c] + f1 * f2 * P11[c];
      s.samp[k][c] = v;
      s.f[c] *= v;
    }
  }
  for (int o = 0; o < kHidden; ++o) {
    double acc = df.b1[o];
    for (int c = 0; c < C; ++c) acc += df.w1[o * C + c] * s.f[c];
    s.pre1[o] = acc;
    s.h1[o] = acc > 0 ? acc : 0;
  }
  for (int o = 0; o < kHidden; ++o) {
    double acc = df.b2[o];
    for (int c = 0; c < kHidden; ++c) acc += df.w2[o * kHidden + c] * s.h1[c];
    s.pre2[o] = acc;
    s.h2[o] = acc > 0 ? acc : 0;
  }
  for (int o = 0; o < 11; ++o) {
    double acc = df.bh[o];
    for (int c = 0; c < kHidden; ++c) acc += df.wh[o * kHidden + c] * s.h2[c];
    s.delta[o] = acc;
  }
}

// Gradient-only decisions of the reverse pass that a caller takes the other
// way (all false: the FP64 decisions).  flip_cell at an interior grid node
// differentiates through the neighbouring cell; at a border node it toggles
// the clamp (which zeroes the coordinate's gradient).
struct DeformFlips {
  const bool* relu1;
  const bool* relu2;
  const bool (*cell)[2];
};

// Gradient of the head outputs (ddelta[11]) back to the canonical mean.
void deform_backward(const or_deform& df, const DeformState& s, const double ddelta[11], double dmu[3],
                     const DeformFlips* fl = nullptr) {
  const int C = df.C, R = df.R;
  double dh2[kHidden], dh1[kHidden], dfv[kMaxC];
  for (int c = 0; c < kHidden; ++c) {
    double acc = 0;
    for (int o = 0; o < 11; ++o) acc += df.wh[o * kHidden + c] * ddelta[o];
    const bool on = (s.pre2[c] > 0) != (fl && fl->relu2[c]);
    dh2[c] = on ? acc : 0;
  }
  for (int c = 0; c < kHidden; ++c) {
    double acc = 0;
    for (int o = 0; o < kHidden; ++o) acc += df.w2[o * kHidden + c] * dh2[o];
    const bool on = (s.pre1[c] > 0) != (fl && fl->relu1[c]);
    dh1[c] = on ? acc : 0;
  }
  for (int c = 0; c < C; ++c) {
    double acc = 0;
    for (int o = 0; o < kHidden; ++o) acc += df.w1[o * C + c] * dh1[o];
    dfv[c] = acc;
  }
  double dcoord[4] = {0, 0, 0, 0};
  for (int k = 0; k < 6; ++k) {
    double f1 = s.fr[k][0], f2 = s.fr[k][1];
    int i = s.i0[k][0], j = s.i0[k][1];
    int clamped[2] = {s.clamped[k][0], s.clamped[k][1]};
    for (int e = 0; e < 2; ++e) {
      if (!(fl && fl->cell[k][e])) continue;
      const double gp = s.pos[k][e];
      const int n = (int)std::nearbyint(gp);
      if (n <= 0 || n >= R - 1) {
        clamped[e] = !clamped[e];
      } else {
        int& ie = e == 0 ? i : j;
        double& fe = e == 0 ? f1 : f2;
        ie = ie == n ? n - 1 : n;
        fe = gp - ie;
      }
    }
    const double* P00 = df.planes + ((size_t)(k * R + i) * R + j) * C;
    const double* P10 = df.planes + ((size_t)(k * R + i + 1) * R + j) * C;
    const double* P01 = df.planes + ((size_t)(k * R + i) * R + j + 1) * C;
    const double* P11 = df.planes + ((size_t)(k * R + i + 1) * R + j + 1) * C;
    double dg1 = 0, dg2 = 0;
    for (int c = 0; c < C; ++c) {
      double others = 1.0;  // product of the other five samples
      for (int m = 0; m < 6; ++m)
        if (m != k) others *= s.samp[m][c];
      const double ds = dfv[c] * others;
      dg1 += ds * ((1 - f2) * (P10[c] - P00[c]) + f2 * (P11[c] - P01[c]));
      dg2 += ds * ((1 - f1) * (P01[c] - P00[c]) + f1 * (P11[c] - P10[c]));
    }
    if (!clamped[0]) dcoord[kPair[k][0]] += dg1 * 0.5 * (R - 1);
    if (!clamped[1]) dcoord[kPair[k][1]] += dg2 * 0.5 * (R - 1);
  }
  for (int a = 0; a < 3; ++a) dmu[a] = dcoord[a] * 2.0 / (df.bbox_max[a] - df.bbox_min[a]);
}

// ---------------------------------------------------------------------------
// Per-Gaussian forward state (deformation applied, projected).
// ---------------------------------------------------------------------------
struct GState {
  DeformState ds;
  int has_deform;
  double mu[3];        // deformed mean
  double qt[4], qn;    // q + dq and its norm
  double q[4];         // unit quaternion
  double s[3];         // scales
  double o;            // opacity
  double Rm[9], RS[9], Sig[9];
  double p[3];         // camera-space centre
  double tx, ty, txc, tyc;
  int clx, cly;
  double J[6], T[6];   // 2x3, row-major
  double a, b, c, det; // dilated 2D covariance [[a,b],[b,c]]
  double conic[3];
  double u, v;
  double dir[3], dnorm;
  double Y[16], dY[16][3];
  double rgb_raw[3], rgb[3];
  int radius;
  int rect[4];
  double rmargin;
  double zerr;         // bound on the binary32 error of the camera-space depth
  int gflags;
  int visible;
  double rnear;        // nearest integer to 3 sqrt(lambda_max) (radius-ceil decision)
  // Gradient-only decisions within rounding of their threshold (rgb clamp,
  // J clamp, ReLU, grid cell), in a fixed order: their number, and which of
  // them the reverse pass takes the other way (bit k of gflip flips the
  // k-th).  A binary32 evaluation may take either branch there.
  int gndec;
  uint64_t gflip;
  bool flip_rgb[3], flip_jx, flip_jy;
  bool flip_relu1[kHidden], flip_relu2[kHidden];
  bool flip_cell[6][2];
};

// Records a near-threshold gradient decision; true when gflip takes it the
// other way.
bool gdecision(GState& st) {
  const bool f = ((st.gflip >> st.gndec) & 1ull) != 0;
  ++st.gndec;
  return f;
}

void quat_to_rot(const double q[4], double Rm[9]) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  Rm[0] = 1 - 2 * (y * y + z * z); Rm[1] = 2 * (x * y - w * z); Rm[2] = 2 * (x * z + w * y);
  Rm[3] = 2 * (x * y + w * z); Rm[4] = 1 - 2 * (x * x + z * z); Rm[5] = 2 * (y * z - w * x);
  Rm[6] = 2 * (x * z - w * y); Rm[7] = 2 * (y * z + w * x); Rm[8] = 1 - 2 * (x * x + y * y);
}

void gaussian_forward(const or_scene& sc, const or_deform* df, const or_camera& cam, double t, int g,
                      const double* geps, GState& st, uint64_t gflip = 0) {
  double delta[11] = {0};
  st.gflip = gflip;
  st.has_deform = df && df->enabled;
  if (st.has_deform) {
    deform_forward(*df, sc.means + 3 * g, t, st.ds);
    std::memcpy(delta, st.ds.delta, sizeof(delta));
    if (df->noise)
      for (int a = 0; a < 3; ++a) delta[a] += df->noise_scale * t * df->noise[3 * g + a];
  }
  std::memcpy(st.ds.delta, delta, sizeof(delta));
  st.gflags = 0;
  st.gndec = 0;
  st.flip_rgb[0] = st.flip_rgb[1] = st.flip_rgb[2] = false;
  st.flip_jx = st.flip_jy = false;
  for (int o = 0; o < kHidden; ++o) st.flip_relu1[o] = st.flip_relu2[o] = false;
  for (int k = 0; k < 6; ++k) st.flip_cell[k][0] = st.flip_cell[k][1] = false;
  // Eq. 6 reading: mu + d_mu; quaternion + d_q renormalised; log-scale + d_s;
  // opacity logit + d_o.
  for (int a = 0; a < 3; ++a) st.mu[a] = sc.means[3 * g + a] + delta[a];
  double n2 = 0;
  for (int a = 0; a < 4; ++a) { st.qt[a] = sc.quats[4 * g + a] + delta[3 + a]; n2 += st.qt[a] * st.qt[a]; }
  st.qn = std::sqrt(n2);
  for (int a = 0; a < 4; ++a) st.q[a] = st.qt[a] / st.qn;
  for (int a = 0; a < 3; ++a) st.s[a] = std::exp(sc.log_scales[3 * g + a] + delta[7 + a]);
  st.o = 1.0 / (1.0 + std::exp(-(sc.logits[g] + delta[10])));
  // Eq. 2: Sigma = R S S^T R^T.
  quat_to_rot(st.q, st.Rm);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) st.RS[3 * i + j] = st.Rm[3 * i + j] * st.s[j];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0;
      for (int k = 0; k < 3; ++k) acc += st.RS[3 * i + k] * st.RS[3 * j + k];
      st.Sig[3 * i + j] = acc;
    }
  const double* V = cam.view;
  for (int i = 0; i < 3; ++i)
    st.p[i] = V[4 * i + 0] * st.mu[0] + V[4 * i + 1] * st.mu[1] + V[4 * i + 2] * st.mu[2] + V[4 * i + 3];
  {
    // Standard rounding-error bound of the binary32 depth z = V2 . (mu + dmu) + V23,
    // unit roundoff u = 2^-24: the rounding of each mu + dmu (propagated by
    // |V2a|), a generous bound for the binary32 offsets themselves, one u per
    // product whose factor is not a power of two and per addition of
    // non-zero terms.  Exact operations (factor 0, +-1, additions of zero)
    // contribute nothing.
    const double u = std::ldexp(1.0, -24);
    double prop = 0, sum = 0;
    int inexact = 0, nz = 0;
    for (int a = 0; a < 4; ++a) {
      const double va = V[8 + a];
      const double term = a < 3 ? va * st.mu[a] : va;
      if (term != 0) ++nz;
      sum += std::fabs(term);
      if (a < 3) {
        prop += std::fabs(va) * (std::fabs(st.mu[a]) + 64.0 * std::fabs(delta[a]));
        int ex;
        const double m = std::frexp(std::fabs(va), &ex);
        if (va != 0 && m != 0.5) ++inexact;
      }
    }
    st.zerr = u * (prop + (inexact + std::max(nz - 1, 0)) * sum);
  }
  st.visible = 0;
  st.radius = 0;
  st.rect[0] = 0; st.rect[1] = 0; st.rect[2] = -1; st.rect[3] = -1;
  st.rmargin = 1.0;
  const double z = st.p[2];
  // View-dependent colour (computed for culled Gaussians too; unused there).
  double dv[3];
  for (int a = 0; a < 3; ++a) dv[a] = st.mu[a] - cam.campos[a];
  st.dnorm = std::sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
  for (int a = 0; a < 3; ++a) st.dir[a] = dv[a] / st.dnorm;
  sh_basis(st.dir, st.Y, st.dY);
  const int nb = (sc.sh_degree + 1) * (sc.sh_degree + 1);
  for (int ch = 0; ch < 3; ++ch) {
    double acc = 0.5;
    for (int k = 0; k < nb; ++k) acc += sc.sh[(size_t)g * 48 + 3 * k + ch] * st.Y[k];
    st.rgb_raw[ch] = acc;
    st.rgb[ch] = acc > 0 ? acc : 0;
    if (geps && std::fabs(acc) < geps[0]) {
      st.gflags |= 1;
      st.flip_rgb[ch] = gdecision(st);
    }
  }
  if (!(z > cam.znear)) return;
  // EWA (Eq. 9 of Sec. 3.3) with the affine Jacobian of the pinhole model at
  // the centre; x/z and y/z clamped to 1.3x the half field of view.
  st.tx = st.p[0] / z;
  st.ty = st.p[1] / z;
  const double limx = 1.3 * 0.5 * cam.width / cam.fx, limy = 1.3 * 0.5 * cam.height / cam.fy;
  st.clx = st.tx < -limx || st.tx > limx;
  st.cly = st.ty < -limy || st.ty > limy;
  st.txc = std::min(limx, std::max(-limx, st.tx));
  st.tyc = std::min(limy, std::max(-limy, st.ty));
  if (geps && std::fabs(std::fabs(st.tx) - limx) < geps[1] * limx) {
    st.gflags |= 2;
    st.flip_jx = gdecision(st);
  }
  if (geps && std::fabs(std::fabs(st.ty) - limy) < geps[1] * limy) {
    st.gflags |= 2;
    st.flip_jy = gdecision(st);
  }
  st.J[0] = cam.fx / z; st.J[1] = 0; st.J[2] = -cam.fx * st.txc / z;
  st.J[3] = 0; st.J[4] = cam.fy / z; st.J[5] = -cam.fy * st.tyc / z;
  for (int r = 0; r < 2; ++r)
    for (int j = 0; j < 3; ++j) {
      double acc = 0;
      for (int k = 0; k < 3; ++k) acc += st.J[3 * r + k] * V[4 * k + j];
      st.T[3 * r + j] = acc;
    }
  double S2[4];
  for (int r = 0; r < 2; ++r)
    for (int q = 0; q < 2; ++q) {
      double acc = 0;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) acc += st.T[3 * r + i] * st.Sig[3 * i + j] * st.T[3 * q + j];
      S2[2 * r + q] = acc;
    }
  // Low-pass dilation of 0.3 px^2 on the diagonal (reading).
  st.a = S2[0] + kDilation;
  st.b = S2[1];
  st.c = S2[3] + kDilation;
  st.det = st.a * st.c - st.b * st.b;
  if (!(st.det > 0)) return;
  st.conic[0] = st.c / st.det;
  st.conic[1] = -st.b / st.det;
  st.conic[2] = st.a / st.det;
  const double mid = 0.5 * (st.a + st.c);
  const double lam = mid + std::sqrt(std::max(0.1, mid * mid - st.det));
  const double xr = 3.0 * std::sqrt(lam);
  st.radius = (int)std::ceil(xr);
  st.rnear = std::nearbyint(xr);
  st.rmargin = std::fabs(xr - st.rnear) / xr;
  st.u = cam.fx * st.tx + cam.cx;
  st.v = cam.fy * st.ty + cam.cy;
  st.visible = 1;
  // Pixels whose centre (x+0.5, y+0.5) lies in the square of half-side r.
  const double r = st.radius;
  double x0 = std::ceil(st.u - r - 0.5), x1 = std::floor(st.u + r - 0.5);
  double y0 = std::ceil(st.v - r - 0.5), y1 = std::floor(st.v + r - 0.5);
  x0 = std::max(x0, 0.0); y0 = std::max(y0, 0.0);
  x1 = std::min(x1, (double)cam.width - 1); y1 = std::min(y1, (double)cam.height - 1);
  if (x0 <= x1 && y0 <= y1) {
    st.rect[0] = (int)x0; st.rect[1] = (int)y0; st.rect[2] = (int)x1; st.rect[3] = (int)y1;
  }
  if (geps && st.has_deform) {
    double rms1 = 0, rms2 = 0;
    for (int o = 0; o < kHidden; ++o) { rms1 += st.ds.pre1[o] * st.ds.pre1[o]; rms2 += st.ds.pre2[o] * st.ds.pre2[o]; }
    rms1 = std::sqrt(rms1 / kHidden) + 1e-30; rms2 = std::sqrt(rms2 / kHidden) + 1e-30;
    for (int o = 0; o < kHidden; ++o)
      if (std::fabs(st.ds.pre1[o]) < geps[2] * rms1) {
        st.gflags |= 4;
        st.flip_relu1[o] = gdecision(st);
      }
    for (int o = 0; o < kHidden; ++o)
      if (std::fabs(st.ds.pre2[o]) < geps[2] * rms2) {
        st.gflags |= 4;
        st.flip_relu2[o] = gdecision(st);
      }
    // Only the spatial coordinates carry a gradient (to the canonical mean);
    // the time coordinate of the xt, yt, zt planes does not.
    for (int k = 0; k < 6; ++k)
      for (int e = 0; e < 2; ++e) {
        if (kPair[k][e] == 3) continue;
        const double gp = st.ds.pos[k][e];
        if (std::fabs(gp - std::nearbyint(gp)) < geps[3] * (df->R - 1)) {
          st.gflags |= 8;
          st.flip_cell[k][e] = gdecision(st);
        }
      }
  }
}

// ---------------------------------------------------------------------------
// Per-pixel compositing (Eq. 7-8): candidates are the visible Gaussians whose
// square of half-side r contains the pixel centre, ordered by (depth, index).
// alpha = min(0.99, o exp(power)); skip power > 0 and alpha < 1/255; stop
// before adding a Gaussian that would take T below 1e-4.
// ---------------------------------------------------------------------------
struct Contrib {
  int g;
  double alpha, G, T;  // alpha, exp(power), transmittance before this Gaussian
  double dx, dy;
  int clamped;
};

enum {
  kFlagIncl = 1,    // inclusion square / radius ceil near a decision
  kFlagSkip = 2,    // alpha near 1/255
  kFlagTerm = 4,    // T(1-alpha) near 1e-4
  kFlagDepth = 8,   // near-equal depths among contributors
  kFlagClamp = 16,  // o*G near 0.99 (gradient only)
};

struct PixelResult {
  double rgb[3], depth, alpha, sumw;
  double T;
  int ncontrib, flags;
  uint64_t sig;
  int ndec;  // near-threshold decisions met (see composite_pixel)
};

// Near-threshold decisions of one pixel, counted in the order they are met;
// bit k of `flip` takes the k-th one the other way.
struct PixelDecisions {
  uint64_t flip;
  int n;
  bool take(bool natural) {
    const bool f = ((flip >> n) & 1ull) != 0;
    ++n;
    return natural != f;
  }
};

// Composites pixel (x, y).  With eps, every decision whose FP64 margin is
// inside the binary32 error model is flagged and counted as a decision, in
// this order: (1) inclusion of Gaussians near the edge of their square (by
// index; the other branch puts a Gaussian inside the square out and one
// outside in -- for a radius ceil near an integer n the ring n < m <= n + 1
// is the part that changes); (2) the order of two possible contributors
// (alpha >= 1/255 up to the skip margin) that are adjacent in depth order
// with depths inside their binary32 error bounds (the other branch swaps
// them); (3) per candidate, front to back, the alpha skip and then the
// termination test.  A binary32 evaluation may take either branch of each;
// `flip` (bit k: the k-th decision the other way) selects one of the
// resulting results.  flip = 0 is the FP64 result.
void composite_pixel(const or_scene& sc, const std::vector<GState>& gs, const or_camera& cam, const double* bg,
                     int x, int y, const double* eps, PixelResult& res, double* feat_out,
                     std::vector<Contrib>* contribs, uint64_t flip = 0) {
  (void)cam;
  const double px = x + 0.5, py = y + 0.5;
  const int P = sc.P, D = sc.D;
  std::vector<int> cand;
  int flags = 0;
  PixelDecisions dec{flip, 0};
  for (int g = 0; g < P; ++g) {
    const GState& s = gs[g];
    if (!s.visible) continue;
    const double dx = px - s.u, dy = py - s.v;
    const double m = std::max(std::fabs(dx), std::fabs(dy));
    const double r = s.radius;
    bool in = m <= r;
    if (eps) {
      // An inclusion decision only matters where the Gaussian would contribute.
      const bool near_edge = std::fabs(m - r) < eps[0] * (std::fabs(s.u) + std::fabs(s.v) + r);
      const bool ring = s.rmargin < eps[1] && m > s.rnear && m <= s.rnear + 1.0;
      if (near_edge || ring) {
        const double power = -0.5 * (s.conic[0] * dx * dx + s.conic[2] * dy * dy) - s.conic[1] * dx * dy;
        if (s.o * std::exp(power) >= kAlphaMin * (1 - 1e-3)) {
          flags |= kFlagIncl;
          in = dec.take(in);
        }
      }
    }
    if (in) cand.push_back(g);
  }
  std::sort(cand.begin(), cand.end(), [&](int i, int k) {
    if (gs[i].p[2] != gs[k].p[2]) return gs[i].p[2] < gs[k].p[2];
    return i < k;
  });
  auto alpha_at = [&](int g) {
    const GState& s = gs[g];
    const double dx = px - s.u, dy = py - s.v;
    const double power = -0.5 * (s.conic[0] * dx * dx + s.conic[2] * dy * dy) - s.conic[1] * dx * dy;
    return power > 0 ? 0.0 : std::min(kAlphaMax, s.o * std::exp(power));
  };
  if (eps) {
    // Order decisions among the possible contributors, front to back.
    int prev = -1;
    for (size_t ci = 0; ci < cand.size(); ++ci) {
      if (alpha_at(cand[ci]) < kAlphaMin * (1 - eps[2])) continue;
      if (prev >= 0) {
        const GState& a = gs[cand[prev]];
        const GState& b = gs[cand[ci]];
        if (std::fabs(b.p[2] - a.p[2]) <= eps[4] * (a.zerr + b.zerr) && dec.take(false)) {
          std::swap(cand[prev], cand[ci]);
        }
      }
      prev = (int)ci;
    }
  }
  double T = 1.0, C[3] = {0, 0, 0}, Z = 0, sumw = 0;
  for (int k = 0; k < D; ++k) feat_out[k] = 0;
  int n = 0;
  uint64_t sig = 1469598103934665603ull;
  int prev_contrib = -1;
  for (size_t ci = 0; ci < cand.size(); ++ci) {
    const int g = cand[ci];
    const GState& s = gs[g];
    const double dx = px - s.u, dy = py - s.v;
    const double power = -0.5 * (s.conic[0] * dx * dx + s.conic[2] * dy * dy) - s.conic[1] * dx * dy;
    if (power > 0) continue;
    const double G = std::exp(power);
    const double oG = s.o * G;
    const double alpha = std::min(kAlphaMax, oG);
    bool skip = alpha < kAlphaMin;
    if (eps && std::fabs(alpha - kAlphaMin) < eps[2] * kAlphaMin) {
      flags |= kFlagSkip;
      skip = dec.take(skip);
    }
    if (skip) continue;
    const double Tn = T * (1 - alpha);
    bool stop = Tn < kTMin;
    if (eps && std::fabs(Tn - kTMin) < eps[3] * kTMin) {
      flags |= kFlagTerm;
      stop = dec.take(stop);
    }
    if (stop) break;
    if (eps && std::fabs(oG - kAlphaMax) < eps[5] * kAlphaMax) flags |= kFlagClamp;
    if (eps && prev_contrib >= 0) {
      // Two depths closer than their binary32 error bounds (times eps[4]) may
      // be ordered either way.
      const double d0 = gs[prev_contrib].p[2], d1 = s.p[2];
      if (std::fabs(d1 - d0) <= eps[4] * (gs[prev_contrib].zerr + s.zerr)) flags |= kFlagDepth;
    }
    prev_contrib = g;
    const double w = alpha * T;
    for (int ch = 0; ch < 3; ++ch) C[ch] += w * s.rgb[ch];
    Z += w * s.p[2];
    const double* z = sc.feat + (size_t)g * D;
    for (int k = 0; k < D; ++k) feat_out[k] += w * z[k];
    sumw += w;
    if (contribs) contribs->push_back(Contrib{g, alpha, G, T, dx, dy, oG > kAlphaMax});
    T = Tn;
    ++n;
    sig = (sig ^ (uint64_t)(g + 1) * 0x9E3779B97F4A7C15ull) * 1099511628211ull;
    sig ^= (uint64_t)(oG > kAlphaMax);
  }
  for (int ch = 0; ch < 3; ++ch) res.rgb[ch] = C[ch] + T * bg[ch];
  res.depth = Z;
  res.alpha = 1 - T;
  res.sumw = sumw;
  res.T = T;
  res.ncontrib = n;
  res.flags = flags;
  res.sig = sig;
  res.ndec = dec.n;
}

void fill_gauss_out(const std::vector<GState>& gs, or_gauss* out) {
  const int P = (int)gs.size();
  for (int g = 0; g < P; ++g) {
    const GState& s = gs[g];
    if (out->delta) for (int k = 0; k < 11; ++k) out->delta[11 * g + k] = s.ds.delta[k];
    if (out->uv) { out->uv[2 * g] = s.visible ? s.u : 0; out->uv[2 * g + 1] = s.visible ? s.v : 0; }
    if (out->conic) for (int k = 0; k < 3; ++k) out->conic[3 * g + k] = s.visible ? s.conic[k] : 0;
    if (out->opacity) out->opacity[g] = s.o;
    if (out->depth) out->depth[g] = s.p[2];
    if (out->rgb) for (int k = 0; k < 3; ++k) out->rgb[3 * g + k] = s.rgb[k];
    if (out->rgb_raw) for (int k = 0; k < 3; ++k) out->rgb_raw[3 * g + k] = s.rgb_raw[k];
    if (out->radius) out->radius[g] = s.radius;
    if (out->rect) for (int k = 0; k < 4; ++k) out->rect[4 * g + k] = s.rect[k];
    if (out->rmargin) out->rmargin[g] = s.rmargin;
    if (out->gflags) out->gflags[g] = s.gflags;
    if (out->gndec) out->gndec[g] = s.gndec;
  }
}

void all_gaussians(const or_scene& sc, const or_deform* df, const or_camera& cam, double t, const double* geps,
                   std::vector<GState>& gs, const uint64_t* gflip = nullptr) {
  gs.resize(sc.P);
#pragma omp parallel for schedule(dynamic, 256)
  for (int g = 0; g < sc.P; ++g) gaussian_forward(sc, df, cam, t, g, geps, gs[g], gflip ? gflip[g] : 0);
}

// ---------------------------------------------------------------------------
// Reverse pass of one Gaussian's preprocess: screen-space gradients
// (du, dv, dconic a/b/c, dopacity, drgb[3], ddepth) -> canonical parameters.
// ---------------------------------------------------------------------------
void gaussian_backward(const or_scene& sc, const or_deform* df, const or_camera& cam, const GState& s,
                       const double* sg, int g, double* d_means, double* d_log_scales, double* d_quats,
                       double* d_logits, double* d_sh) {
  const double du = sg[0], dv = sg[1];
  const double dA = sg[2], dB = sg[3], dC = sg[4];
  const double dop = sg[5];
  const double* drgb = sg + 6;
  const double ddepth = sg[9];
  const double* V = cam.view;
  double dmu[3] = {0, 0, 0};
  double dp[3] = {0, 0, 0};
  // Colour: rgb = max(0, sum sh*Y + 0.5); gradient passes where raw >= 0.
  const int nb = (sc.sh_degree + 1) * (sc.sh_degree + 1);
  double ddir[3] = {0, 0, 0};
  for (int ch = 0; ch < 3; ++ch) {
    const double gch = (s.rgb_raw[ch] >= 0) != s.flip_rgb[ch] ? drgb[ch] : 0.0;
    for (int k = 0; k < 16; ++k) {
      const double v = k < nb ? gch * s.Y[k] : 0.0;
      d_sh[(size_t)g * 48 + 3 * k + ch] = v;
      if (k < nb)
        for (int a = 0; a < 3; ++a) ddir[a] += gch * sc.sh[(size_t)g * 48 + 3 * k + ch] * s.dY[k][a];
    }
  }
  const double dd = ddir[0] * s.dir[0] + ddir[1] * s.dir[1] + ddir[2] * s.dir[2];
  for (int a = 0; a < 3; ++a) dmu[a] += (ddir[a] - s.dir[a] * dd) / s.dnorm;
  // Opacity through the sigmoid.
  const double dlogit = dop * s.o * (1 - s.o);
  double dlogs[3] = {0, 0, 0};
  double dqt[4] = {0, 0, 0, 0};
  if (s.visible) {
    const double z = s.p[2];
    // Conic = inverse of [[a,b],[b,c]]: dSigma' = -M G M with G the symmetric
    // gradient of M = [[A,B],[B,C]] (B appears twice in the quadratic form).
    const double M[4] = {s.conic[0], s.conic[1], s.conic[1], s.conic[2]};
    const double Gm[4] = {dA, 0.5 * dB, 0.5 * dB, dC};
    double MG[4], Gs[4];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) MG[2 * i + j] = M[2 * i] * Gm[j] + M[2 * i + 1] * Gm[2 + j];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) Gs[2 * i + j] = -(MG[2 * i] * M[j] + MG[2 * i + 1] * M[2 + j]);
    // Sigma' = T Sigma T^T: dSigma = T^T Gs T, dT = 2 Gs T Sigma.
    double dSig[9], dT[6];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double acc = 0;
        for (int r = 0; r < 2; ++r)
          for (int q = 0; q < 2; ++q) acc += s.T[3 * r + i] * Gs[2 * r + q] * s.T[3 * q + j];
        dSig[3 * i + j] = acc;
      }
    for (int r = 0; r < 2; ++r)
      for (int j = 0; j < 3; ++j) {
        double acc = 0;
        for (int q = 0; q < 2; ++q)
          for (int k = 0; k < 3; ++k) acc += Gs[2 * r + q] * s.T[3 * q + k] * s.Sig[3 * k + j];
        dT[3 * r + j] = 2 * acc;
      }
    // T = J W: dJ = dT W^T.
    double dJ[6];
    for (int r = 0; r < 2; ++r)
      for (int k = 0; k < 3; ++k) {
        double acc = 0;
        for (int j = 0; j < 3; ++j) acc += dT[3 * r + j] * V[4 * k + j];
        dJ[3 * r + k] = acc;
      }
    // J = [[fx/z, 0, -fx txc/z], [0, fy/z, -fy tyc/z]].
    dp[2] += -cam.fx / (z * z) * dJ[0] - cam.fy / (z * z) * dJ[4];
    dp[2] += cam.fx * s.txc / (z * z) * dJ[2] + cam.fy * s.tyc / (z * z) * dJ[5];
    double dtxc = -cam.fx / z * dJ[2], dtyc = -cam.fy / z * dJ[5];
    double dtx = (s.clx != 0) != s.flip_jx ? 0.0 : dtxc, dty = (s.cly != 0) != s.flip_jy ? 0.0 : dtyc;
    // Projected centre u = fx x/z + cx, v = fy y/z + cy.
    dtx += cam.fx * du;
    dty += cam.fy * dv;
    dp[0] += dtx / z;
    dp[1] += dty / z;
    dp[2] += -s.p[0] / (z * z) * dtx - s.p[1] / (z * z) * dty;
    dp[2] += ddepth;
    for (int a = 0; a < 3; ++a) dmu[a] += V[0 * 4 + a] * dp[0] + V[1 * 4 + a] * dp[1] + V[2 * 4 + a] * dp[2];
    // Sigma = (RS)(RS)^T: d(RS) = 2 dSigma RS.
    double dRS[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double acc = 0;
        for (int k = 0; k < 3; ++k) acc += (dSig[3 * i + k] + dSig[3 * k + i]) * s.RS[3 * k + j];
        dRS[3 * i + j] = acc;
      }
    double dR[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) dR[3 * i + j] = dRS[3 * i + j] * s.s[j];
    for (int j = 0; j < 3; ++j) {
      double acc = 0;
      for (int i = 0; i < 3; ++i) acc += dRS[3 * i + j] * s.Rm[3 * i + j];
      dlogs[j] = acc * s.s[j];
    }
    const double w = s.q[0], x = s.q[1], y = s.q[2], zq = s.q[3];
    double dq[4];
    dq[0] = 2 * (-zq * dR[1] + y * dR[2] + zq * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
    dq[1] = 2 * (y * dR[1] + zq * dR[2] + y * dR[3] - 2 * x * dR[4] - w * dR[5] + zq * dR[6] + w * dR[7] - 2 * x * dR[8]);
    dq[2] = 2 * (-2 * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + zq * dR[5] - w * dR[6] + zq * dR[7] - 2 * y * dR[8]);
    dq[3] = 2 * (-2 * zq * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2 * zq * dR[4] + y * dR[5] + x * dR[6] + y * dR[7]);
    const double qd = dq[0] * s.q[0] + dq[1] * s.q[1] + dq[2] * s.q[2] + dq[3] * s.q[3];
    for (int a = 0; a < 4; ++a) dqt[a] = (dq[a] - s.q[a] * qd) / s.qn;
  }
  // Canonical parameters receive the gradient of the deformed ones directly
  // (mu' = mu + d_mu, ...), plus the path through the HexPlane grid.
  double dmu_total[3] = {dmu[0], dmu[1], dmu[2]};
  if (s.has_deform) {
    double ddelta[11];
    for (int a = 0; a < 3; ++a) ddelta[a] = dmu[a];
    for (int a = 0; a < 4; ++a) ddelta[3 + a] = dqt[a];
    for (int a = 0; a < 3; ++a) ddelta[7 + a] = dlogs[a];
    ddelta[10] = dlogit;
    double dgrid[3];
    const DeformFlips fl{s.flip_relu1, s.flip_relu2, s.flip_cell};
    deform_backward(*df, s.ds, ddelta, dgrid, &fl);
    for (int a = 0; a < 3; ++a) dmu_total[a] += dgrid[a];
  }
  for (int a = 0; a < 3; ++a) d_means[3 * g + a] = dmu_total[a];
  for (int a = 0; a < 3; ++a) d_log_scales[3 * g + a] = dlogs[a];
  for (int a = 0; a < 4; ++a) d_quats[4 * g + a] = dqt[a];
  d_logits[g] = dlogit;
}

}  // namespace

extern "C" {

// Per-Gaussian deformation + projection + colour for all P Gaussians.
// geps (may be NULL): thresholds of the gradient-affecting decisions
// {rgb clamp |raw|, J clamp (relative), relu (relative to rms), grid cell}.
int or_preprocess(const or_scene* sc, const or_deform* df, const or_camera* cam, double t, const double* geps,
                  or_gauss* out) {
  if (!sc || !cam || !out || sc->D > kMaxD || (df && df->enabled && df->C > kMaxC)) return 1;
  std::vector<GState> gs;
  all_gaussians(*sc, df, *cam, t, geps, gs);
  fill_gauss_out(gs, out);
  return 0;
}

// Composite the listed pixels (pix = npix (x,y) pairs).  eps (may be NULL):
// decision thresholds {inclusion (relative to |u|+|v|+r), radius ceil
// (relative), alpha skip (relative), termination (relative), depth tie
// (safety factor on the two depths' binary32 error bounds), alpha clamp
// (relative)}.  Outputs per pixel: rgb[3]
// (with bg*T), depth, alpha = 1-T, feat[D], sumw (sum of blend weights),
// ncontrib, flags, sig (hash of the contributor sequence).
int or_render(const or_scene* sc, const or_deform* df, const or_camera* cam, double t, const double* bg,
              int npix, const int* pix, const double* eps, double* out_rgb, double* out_depth, double* out_alpha,
              double* out_feat, double* out_sumw, int* out_ncontrib, int* out_flags, uint64_t* out_sig) {
  if (!sc || !cam || sc->D > kMaxD || (df && df->enabled && df->C > kMaxC)) return 1;
  std::vector<GState> gs;
  all_gaussians(*sc, df, *cam, t, nullptr, gs);
  const int D = sc->D;
#pragma omp parallel for schedule(dynamic, 16)
  for (int i = 0; i < npix; ++i) {
    PixelResult r;
    std::vector<double> f(D > 0 ? D : 1);
    composite_pixel(*sc, gs, *cam, bg, pix[2 * i], pix[2 * i + 1], eps, r, f.data(), nullptr);
    for (int ch = 0; ch < 3; ++ch) out_rgb[3 * i + ch] = r.rgb[ch];
    out_depth[i] = r.depth;
    out_alpha[i] = r.alpha;
    for (int k = 0; k < D; ++k) out_feat[(size_t)i * D + k] = f[k];
    if (out_sumw) out_sumw[i] = r.sumw;
    if (out_ncontrib) out_ncontrib[i] = r.ncontrib;
    if (out_flags) out_flags[i] = r.flags;
    if (out_sig) out_sig[i] = r.sig;
  }
  return 0;
}

// Every result a binary32 evaluation may legitimately produce at each listed
// pixel: the pixel is composited once per combination of its near-threshold
// decisions (composite_pixel, eps required), at most 2^max_bits
// combinations, and the distinct results (by contributor sequence) are
// written, the FP64 one (flip = 0) first.  Per pixel i and result a <
// max_alts: rgb [i][a][3] (with bg T), depth, alpha, feat [i][a][D], the
// flip mask that produced it; nalts[i] = number written; ndec[i] = decisions
// met by the FP64 result.
int or_render_alts(const or_scene* sc, const or_deform* df, const or_camera* cam, double t, const double* bg,
                   int npix, const int* pix, const double* eps, int max_bits, int max_alts, double* out_rgb,
                   double* out_depth, double* out_alpha, double* out_feat, uint64_t* out_flip, int* out_nalts,
                   int* out_ndec) {
  if (!sc || !cam || !eps || sc->D > kMaxD || (df && df->enabled && df->C > kMaxC) || max_alts < 1 ||
      max_bits < 0 || max_bits > 16)
    return 1;
  std::vector<GState> gs;
  all_gaussians(*sc, df, *cam, t, nullptr, gs);
  const int D = sc->D;
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < npix; ++i) {
    std::vector<double> f(D > 0 ? D : 1);
    std::vector<uint64_t> sigs;
    int seen = 0, na = 0, ndec0 = 0;
    for (uint64_t mask = 0; mask < (1ull << std::min(seen, max_bits)) || mask == 0; ++mask) {
      PixelResult r;
      composite_pixel(*sc, gs, *cam, bg, pix[2 * i], pix[2 * i + 1], eps, r, f.data(), nullptr, mask);
      if (mask == 0) ndec0 = r.ndec;
      seen = std::max(seen, r.ndec);
      // Bits past the decisions this combination met change nothing.
      if (r.ndec < 64 && (mask >> r.ndec) != 0) continue;
      if (std::find(sigs.begin(), sigs.end(), r.sig) != sigs.end()) continue;
      sigs.push_back(r.sig);
      if (na < max_alts) {
        const size_t a = (size_t)i * max_alts + na;
        for (int ch = 0; ch < 3; ++ch) out_rgb[3 * a + ch] = r.rgb[ch];
        out_depth[a] = r.depth;
        out_alpha[a] = r.alpha;
        for (int k = 0; k < D; ++k) out_feat[a * D + k] = f[k];
        out_flip[a] = mask;
        ++na;
      }
    }
    out_nalts[i] = na;
    out_ndec[i] = ndec0;
  }
  return 0;
}

// Gradients of L = sum over the listed pixels of
//   g_rgb . rgb + g_depth * depth + g_alpha * alpha + g_feat . feat
// with respect to every canonical parameter (overwritten, all P rows).
// Upstream arrays are per listed pixel: g_rgb [npix,3], g_depth/g_alpha
// [npix], g_feat [npix,D].
// d_uv (optional, [P][2]): the gradient of the loss with respect to each
// Gaussian's projected centre (u, v) in pixels.
// Decision overrides (all optional): flip [npix] with eps takes pixel i's
// near-threshold decisions the other way as in or_render_alts; gflip [P]
// with geps takes Gaussian g's near-threshold gradient-only decisions (rgb
// clamp, J clamp, ReLU, grid cell; counted by or_preprocess's gndec) the
// other way, bit k for the k-th.
int or_backward(const or_scene* sc, const or_deform* df, const or_camera* cam, double t, const double* bg,
                int npix, const int* pix, const double* g_rgb, const double* g_depth, const double* g_alpha,
                const double* g_feat, double* d_means, double* d_log_scales, double* d_quats, double* d_logits,
                double* d_sh, double* d_feat, double* d_uv, const double* eps, const uint64_t* flip,
                const double* geps, const uint64_t* gflip) {
  if (!sc || !cam || sc->D > kMaxD || (df && df->enabled && df->C > kMaxC)) return 1;
  if ((flip && !eps) || (gflip && !geps)) return 1;
  const int P = sc->P, D = sc->D;
  const int NS = 10;  // du dv dA dB dC dop drgb[3] ddepth
  std::vector<GState> gs;
  all_gaussians(*sc, df, *cam, t, gflip ? geps : nullptr, gs, gflip);
  struct PixGrad { int g; double w; double v[NS]; };
  std::vector<std::vector<PixGrad>> per_pix(npix);
#pragma omp parallel for schedule(dynamic, 16)
  for (int i = 0; i < npix; ++i) {
    PixelResult r;
    std::vector<double> f(D > 0 ? D : 1);
    std::vector<Contrib> cs;
    composite_pixel(*sc, gs, *cam, bg, pix[2 * i], pix[2 * i + 1], flip ? eps : nullptr, r, f.data(), &cs,
                    flip ? flip[i] : 0);
    const double* gr = g_rgb + 3 * i;
    const double* gf = g_feat + (size_t)i * D;
    const double gz = g_depth[i], ga = g_alpha[i];
    const double Tf = r.T;
    // Reverse replay: Q accumulates sum_{k>i} w_k s_k plus the background term,
    // where s_k = g_rgb.c_k + g_depth*depth_k + g_feat.z_k.
    double Q = (gr[0] * bg[0] + gr[1] * bg[1] + gr[2] * bg[2]) * Tf;
    std::vector<PixGrad> out(cs.size());
    for (int ci = (int)cs.size() - 1; ci >= 0; --ci) {
      const Contrib& c = cs[ci];
      const GState& s = gs[c.g];
      const double* z = sc->feat + (size_t)c.g * D;
      const double w = c.alpha * c.T;
      double sdot = gr[0] * s.rgb[0] + gr[1] * s.rgb[1] + gr[2] * s.rgb[2] + gz * s.p[2];
      for (int k = 0; k < D; ++k) sdot += gf[k] * z[k];
      // d out / d alpha_i = T_i x_i - (sum_{k>i} x_k w_k + bg T_final)/(1 - alpha_i);
      // d (1 - T_final) / d alpha_i = T_final / (1 - alpha_i).
      const double dalpha = c.T * sdot - Q / (1 - c.alpha) + ga * Tf / (1 - c.alpha);
      Q += w * sdot;
      PixGrad& pg = out[ci];
      pg.g = c.g;
      pg.w = w;
      for (int k = 0; k < NS; ++k) pg.v[k] = 0;
      if (!c.clamped) {
        const double dpow = dalpha * c.alpha;
        const double A = s.conic[0], B = s.conic[1], Cc = s.conic[2];
        // power = -0.5 (A dx^2 + C dy^2) - B dx dy with dx = px - u, dy = py - v.
        pg.v[0] = dpow * (A * c.dx + B * c.dy);
        pg.v[1] = dpow * (Cc * c.dy + B * c.dx);
        pg.v[2] = dpow * (-0.5 * c.dx * c.dx);
        pg.v[3] = dpow * (-c.dx * c.dy);
        pg.v[4] = dpow * (-0.5 * c.dy * c.dy);
        pg.v[5] = dalpha * c.G;
      }
      for (int ch = 0; ch < 3; ++ch) pg.v[6 + ch] = w * gr[ch];
      pg.v[9] = w * gz;
    }
    per_pix[i].swap(out);
  }
  // Fixed-order accumulation: pixel order, then front-to-back order.
  std::vector<double> sg((size_t)P * NS, 0.0);
  for (size_t k = 0; k < (size_t)P * D; ++k) d_feat[k] = 0;
  for (int i = 0; i < npix; ++i) {
    const double* gf = g_feat + (size_t)i * D;
    for (const PixGrad& pg : per_pix[i]) {
      for (int k = 0; k < NS; ++k) sg[(size_t)pg.g * NS + k] += pg.v[k];
      double* dz = d_feat + (size_t)pg.g * D;
      for (int k = 0; k < D; ++k) dz[k] += pg.w * gf[k];
    }
  }
#pragma omp parallel for schedule(dynamic, 256)
  for (int g = 0; g < P; ++g)
    gaussian_backward(*sc, df, *cam, gs[g], &sg[(size_t)g * NS], g, d_means, d_log_scales, d_quats, d_logits, d_sh);
  if (d_uv)
    for (int g = 0; g < P; ++g) {
      d_uv[2 * g] = sg[(size_t)g * NS];
      d_uv[2 * g + 1] = sg[(size_t)g * NS + 1];
    }
  return 0;
}

// Per-Gaussian state only (deformation offsets, projection, colour,
// radius, pixel rect, radius-ceil margin, gradient decision flags).
int or_gaussians(const or_scene* sc, const or_deform* df, const or_camera* cam, double t, const double* geps,
                 or_gauss* out) {
  return or_preprocess(sc, df, cam, t, geps, out);
}

// Integer stage, binary32 inputs: tile lists sorted by (tile, depth).
// For each Gaussian g with radius > 0 and finite centre: the pixel rect is
// [ceil(u-(r+0.5)), floor(u+(r-0.5))] x [ceil(v-(r+0.5)), floor(v+(r-0.5))]
// clamped to the image, evaluated in binary32 (one rounding per +/-); its
// tiles are emitted row-major with key (tile << 32) | bits(depth), value g;
// a stable sort by key orders each tile by depth and ties by index.
// ranges[2*tile] = start, ranges[2*tile+1] = end.
int or_tile_bin(int P, const float* uv, const int* radius, const float* depth, int W, int H, int tw, int th,
                long long cap, unsigned long long* keys, unsigned int* vals, unsigned int* ranges, long long* K) {
  const int tiles_x = (W + tw - 1) / tw, tiles_y = (H + th - 1) / th;
  std::vector<std::pair<unsigned long long, unsigned int>> list;
  for (int g = 0; g < P; ++g) {
    const int r = radius[g];
    if (r <= 0) continue;
    const float u = uv[2 * g], v = uv[2 * g + 1];
    if (!std::isfinite(u) || !std::isfinite(v)) continue;
    volatile float rf = (float)r;
    volatile float rp = rf + 0.5f, rm = rf - 0.5f;
    volatile float xl = u - rp, xh = u + rm, yl = v - rp, yh = v + rm;
    float x0 = std::ceil((float)xl), x1 = std::floor((float)xh);
    float y0 = std::ceil((float)yl), y1 = std::floor((float)yh);
    x0 = std::max(x0, 0.0f); y0 = std::max(y0, 0.0f);
    x1 = std::min(x1, (float)(W - 1)); y1 = std::min(y1, (float)(H - 1));
    if (!(x0 <= x1 && y0 <= y1)) continue;
    const int tx0 = (int)x0 / tw, tx1 = (int)x1 / tw, ty0 = (int)y0 / th, ty1 = (int)y1 / th;
    unsigned int db;
    std::memcpy(&db, &depth[g], 4);
    for (int ty = ty0; ty <= ty1; ++ty)
      for (int tx = tx0; tx <= tx1; ++tx)
        list.push_back({((unsigned long long)(ty * tiles_x + tx) << 32) | db, (unsigned int)g});
  }
  std::stable_sort(list.begin(), list.end(),
                   [](const std::pair<unsigned long long, unsigned int>& a,
                      const std::pair<unsigned long long, unsigned int>& b) { return a.first < b.first; });
  *K = (long long)list.size();
  if (!keys || !vals || !ranges) return 0;  // size query
  if ((long long)list.size() > cap) return 2;
  for (size_t i = 0; i < list.size(); ++i) { keys[i] = list[i].first; vals[i] = list[i].second; }
  for (int t = 0; t < tiles_x * tiles_y; ++t) { ranges[2 * t] = 0; ranges[2 * t + 1] = 0; }
  for (size_t i = 0; i < list.size(); ++i) {
    const unsigned int t = (unsigned int)(list[i].first >> 32);
    if (i == 0 || (unsigned int)(list[i - 1].first >> 32) != t) ranges[2 * t] = (unsigned int)i;
    if (i + 1 == list.size() || (unsigned int)(list[i + 1].first >> 32) != t) ranges[2 * t + 1] = (unsigned int)(i + 1);
  }
  return 0;
}

// Real SH basis at n unit directions: Y [n,16], dY [n,16,3].
int or_sh_eval(int n, const double* dirs, double* Y, double* dY) {
  for (int i = 0; i < n; ++i) {
    double y[16], dy[16][3];
    sh_basis(dirs + 3 * i, y, dy);
    for (int k = 0; k < 16; ++k) {
      Y[16 * i + k] = y[k];
      for (int a = 0; a < 3; ++a) dY[(16 * i + k) * 3 + a] = dy[k][a];
    }
  }
  return 0;
}

// HexPlane feature f [n,C] and head output delta [n,11] (without the noise
// term) at n canonical means, time t.
int or_deform_eval(const or_deform* df, int n, const double* mu, double t, double* f, double* delta) {
  if (!df || df->C > kMaxC) return 1;
  for (int i = 0; i < n; ++i) {
    DeformState s;
    deform_forward(*df, mu + 3 * i, t, s);
    for (int c = 0; c < df->C; ++c) f[(size_t)i * df->C + c] = s.f[c];
    for (int k = 0; k < 11; ++k) delta[11 * i + k] = s.delta[k];
  }
  return 0;
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
