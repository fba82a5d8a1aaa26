// Plain, slow FP64 CPU oracle for one 3DGS^2-TR iteration.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path links or calls this
// file; only the tests, the package's smoke check and the benchmark's CPU
// baseline leg do.  It shares no code, header, table or constant with the CUDA
// library: every formula below is written out again from the paper and from the
// 3DGS conventions it defers to.
//
// What it computes, and where each piece comes from:
//   * Gaussian primitive and its parameters: Sec. 3.1, Eq. (gaussian-primitive).
//   * EWA projection, SH colour, tile binning and depth order: Sec. 3.1 (the
//     tile-based rasteriser the paper defers to 3DGS).
//   * Alpha blending C = sum_i c_i a_i T_i, T_i = prod_{j<i}(1 - a_j): Sec. 3.1.
//   * Least-squares objective f = 1/(2m) ||F||^2 with F = sqrt(|residual|):
//     Sec. 3.2, Eq. (objective); gradient g = (1/m) J^T F: Sec. 4.1.
//   * Hutchinson diagonal D = (1/m)(1/nu) sum_k z_k . (J^T J z_k): Sec. 4.1.
//   * Algorithm 1 (EMA of g and D, Newton step, clip, update).
//   * Squared Hellinger distance and the per-parameter radii: Sec. 4.2 and
//     Appendix B (mean, scale, opacity, colour, rotation bounds).
//
// Precision: FP64 everywhere, except the tile rectangle of a splat, whose
// integer result is decided in FP32 exactly as the GPU decides it (the inputs of
// that decision are FP32 values).  Forward-mode derivatives use a one-tangent
// dual number; the reverse pass of the blend is written out by hand.
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -fPIC -shared.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <map>
#include <vector>

namespace {

// ---------------------------------------------------------------- dual numbers
struct Dual {
  double v, d;
  Dual(double v_ = 0.0, double d_ = 0.0) : v(v_), d(d_) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual exp(Dual a) {
  double e = std::exp(a.v);
  return Dual(e, e * a.d);
}
inline Dual sqrt(Dual a) {
  double s = std::sqrt(a.v);
  return Dual(s, a.d / (2.0 * s));
}
inline double exp(double a) { return std::exp(a); }
inline double sqrt(double a) { return std::sqrt(a); }
inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }

const double kPi = 3.14159265358979323846;

// ------------------------------------------------------------------- cameras
struct Cam {
  double R[3][3], t[3];
  double fx, fy, cx, cy, znear;
  int W, H;
  double pos[3];  // camera centre in world coordinates, -R^T t
};

// 24 doubles per camera: viewmat[16] (row-major world->camera), fx, fy, cx, cy,
// near, width, height, unused.
Cam make_cam(const double* c) {
  Cam k;
  for (int r = 0; r < 3; ++r) {
    for (int q = 0; q < 3; ++q) k.R[r][q] = c[4 * r + q];
    k.t[r] = c[4 * r + 3];
  }
  k.fx = c[16]; k.fy = c[17]; k.cx = c[18]; k.cy = c[19]; k.znear = c[20];
  k.W = (int)c[21]; k.H = (int)c[22];
  for (int q = 0; q < 3; ++q)
    k.pos[q] = -(k.R[0][q] * k.t[0] + k.R[1][q] * k.t[1] + k.R[2][q] * k.t[2]);
  return k;
}

// ------------------------------------------------------------- parameters
// Row layout of the parameter matrix (rows x pitch):
//   0..2 mean, 3..5 log-scale, 6..9 quaternion (x,y,z,w), 10 opacity logit,
//   11 + 3k + c: SH coefficient k of colour channel c.
const int kRowSH = 11;
inline int n_coeffs(int deg) { return (deg + 1) * (deg + 1); }
inline int n_rows(int deg) { return kRowSH + 3 * n_coeffs(deg); }

template <class S>
struct G3 {
  S mu[3], ls[3], q[4], ol;
  S sh[16][3];
  int K;
};

// Parameters of Gaussian i; if `tan` is given, row r carries tangent tan[r].
template <class S>
G3<S> load_gaussian(const double* P, long pitch, long i, int deg, const double* tan) {
  G3<S> g;
  g.K = n_coeffs(deg);
  auto get = [&](int r) -> S {
    double v = P[(long)r * pitch + i];
    if constexpr (std::is_same<S, Dual>::value) return Dual(v, tan ? tan[r] : 0.0);
    else return v;
  };
  for (int a = 0; a < 3; ++a) { g.mu[a] = get(a); g.ls[a] = get(3 + a); }
  for (int a = 0; a < 4; ++a) g.q[a] = get(6 + a);
  g.ol = get(10);
  for (int k = 0; k < g.K; ++k)
    for (int c = 0; c < 3; ++c) g.sh[k][c] = get(kRowSH + 3 * k + c);
  return g;
}

// --------------------------------------------------------------- SH basis
// Real spherical harmonics up to degree 3 in the 3DGS sign convention, written
// from their normalisation constants sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) times the
// Cartesian polynomials.
template <class S>
void sh_basis(int deg, S x, S y, S z, S* Y) {
  const double c0 = 0.5 * std::sqrt(1.0 / kPi);
  const double c1 = std::sqrt(3.0 / (4.0 * kPi));
  const double c2a = 0.5 * std::sqrt(15.0 / kPi);
  const double c2b = 0.25 * std::sqrt(5.0 / kPi);
  const double c2c = 0.25 * std::sqrt(15.0 / kPi);
  const double c3a = 0.25 * std::sqrt(35.0 / (2.0 * kPi));
  const double c3b = 0.5 * std::sqrt(105.0 / kPi);
  const double c3c = 0.25 * std::sqrt(21.0 / (2.0 * kPi));
  const double c3d = 0.25 * std::sqrt(7.0 / kPi);
  const double c3e = 0.25 * std::sqrt(105.0 / kPi);
  Y[0] = S(c0);
  if (deg < 1) return;
  Y[1] = -c1 * y;
  Y[2] = c1 * z;
  Y[3] = -c1 * x;
  if (deg < 2) return;
  S xx = x * x, yy = y * y, zz = z * z;
  Y[4] = c2a * (x * y);
  Y[5] = -c2a * (y * z);
  Y[6] = c2b * (2.0 * zz - xx - yy);
  Y[7] = -c2a * (x * z);
  Y[8] = c2c * (xx - yy);
  if (deg < 3) return;
  Y[9] = -c3a * y * (3.0 * xx - yy);
  Y[10] = c3b * (x * y * z);
  Y[11] = -c3c * y * (4.0 * zz - xx - yy);
  Y[12] = c3d * z * (2.0 * zz - 3.0 * xx - 3.0 * yy);
  Y[13] = -c3c * x * (4.0 * zz - xx - yy);
  Y[14] = c3e * z * (xx - yy);
  Y[15] = -c3a * x * (xx - 3.0 * yy);
}

// ---------------------------------------------------------- rotation matrix
// Rotation of the normalised quaternion (x, y, z, w), Appendix B.
template <class S>
void rotmat(const S q[4], S R[3][3]) {
  S r = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  S x = q[0] / r, y = q[1] / r, z = q[2] / r, w = q[3] / r;
  R[0][0] = 1.0 - 2.0 * (y * y + z * z);
  R[0][1] = 2.0 * (x * y - w * z);
  R[0][2] = 2.0 * (x * z + w * y);
  R[1][0] = 2.0 * (x * y + w * z);
  R[1][1] = 1.0 - 2.0 * (z * z + x * x);
  R[1][2] = 2.0 * (y * z - w * x);
  R[2][0] = 2.0 * (x * z - w * y);
  R[2][1] = 2.0 * (y * z + w * x);
  R[2][2] = 1.0 - 2.0 * (x * x + y * y);
}

// ------------------------------------------------------------- projection
template <class S>
struct Splat {
  bool valid = false;  // in front of the near plane with a positive-definite 2-D covariance
  S mx, my, A, B, C, o, rgb[3], depth;
  double radius_raw = 0.0;  // 3 sqrt(lambda_max), before rounding up
  int radius = 0;
  int flags = 0;  // bits 0..2: colour channel clamped at 0; bit 3/4: x/y slope clamped
};

// EWA projection of one Gaussian (3DGS conventions, to which Sec. 3.1 defers):
//   Sigma = R diag(s^2) R^T, t = W mu + t_w, J the perspective Jacobian with the
//   image-plane slope clamped at 1.3 x the half field of view,
//   Sigma' = J R_w Sigma R_w^T J^T + 0.3 I, conic = Sigma'^{-1},
//   radius = ceil(3 sqrt(lambda_max(Sigma'))), colour = SH(view dir) + 0.5 >= 0,
//   opacity = sigmoid(logit).
template <class S>
Splat<S> project(const G3<S>& g, const Cam& cam) {
  Splat<S> p;
  S t[3];
  for (int r = 0; r < 3; ++r)
    t[r] = cam.R[r][0] * g.mu[0] + cam.R[r][1] * g.mu[1] + cam.R[r][2] * g.mu[2] + S(cam.t[r]);
  if (val(t[2]) <= cam.znear) return p;

  S R[3][3];
  rotmat(g.q, R);
  S s2[3];
  for (int a = 0; a < 3; ++a) { S s = exp(g.ls[a]); s2[a] = s * s; }
  S Sig[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      Sig[a][b] = R[a][0] * s2[0] * R[b][0] + R[a][1] * s2[1] * R[b][1] + R[a][2] * s2[2] * R[b][2];
  // camera-frame covariance R_w Sigma R_w^T
  S Sc[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      S acc = 0.0;
      for (int u = 0; u < 3; ++u)
        for (int v = 0; v < 3; ++v) acc = acc + cam.R[a][u] * Sig[u][v] * cam.R[b][v];
      Sc[a][b] = acc;
    }
  const double limx = 1.3 * 0.5 * cam.W / cam.fx;
  const double limy = 1.3 * 0.5 * cam.H / cam.fy;
  S u = t[0] / t[2], v = t[1] / t[2];
  S uc = u, vc = v;
  if (val(u) < -limx) uc = S(-limx);
  if (val(u) > limx) uc = S(limx);
  if (val(v) < -limy) vc = S(-limy);
  if (val(v) > limy) vc = S(limy);
  if (std::fabs(val(u)) > limx) p.flags |= 8;
  if (std::fabs(val(v)) > limy) p.flags |= 16;
  S J[2][3];
  J[0][0] = cam.fx / t[2]; J[0][1] = S(0.0); J[0][2] = -cam.fx * uc / t[2];
  J[1][0] = S(0.0); J[1][1] = cam.fy / t[2]; J[1][2] = -cam.fy * vc / t[2];
  S cov[2][2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      S acc = 0.0;
      for (int x = 0; x < 3; ++x)
        for (int y = 0; y < 3; ++y) acc = acc + J[a][x] * Sc[x][y] * J[b][y];
      cov[a][b] = acc;
    }
  S a = cov[0][0] + 0.3, b = cov[0][1], c = cov[1][1] + 0.3;
  S det = a * c - b * b;
  if (!(val(det) > 0.0)) return p;
  p.A = c / det;
  p.B = -b / det;
  p.C = a / det;
  double mid = 0.5 * (val(a) + val(c));
  double lam = mid + std::sqrt(std::max(0.1, mid * mid - val(det)));
  p.radius_raw = 3.0 * std::sqrt(lam);
  p.radius = (int)std::ceil(p.radius_raw);
  p.mx = cam.fx * u + cam.cx;
  p.my = cam.fy * v + cam.cy;
  p.depth = t[2];

  S d[3];
  for (int q = 0; q < 3; ++q) d[q] = g.mu[q] - S(cam.pos[q]);
  S dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  S Y[16];
  int deg = (int)std::lround(std::sqrt((double)g.K)) - 1;
  sh_basis(deg, d[0] / dn, d[1] / dn, d[2] / dn, Y);
  for (int ch = 0; ch < 3; ++ch) {
    S acc = 0.5;
    for (int k = 0; k < g.K; ++k) acc = acc + Y[k] * g.sh[k][ch];
    p.rgb[ch] = (val(acc) < 0.0) ? S(0.0) : acc;
    if (val(acc) < 0.0) p.flags |= 1 << ch;
  }
  p.o = 1.0 / (1.0 + exp(-g.ol));
  p.valid = true;
  return p;
}

// ---------------------------------------------------------------- binning
// Value of the IEEE half with bits h, as a float (exact).
float half_to_float(uint16_t h) {
  const int e = (h >> 10) & 31, m = h & 1023;
  float v;
  if (e == 31)
    v = m ? NAN : INFINITY;
  else if (e == 0)
    v = std::ldexp((float)m, -24);
  else
    v = std::ldexp((float)(m | 1024), e - 25);
  return (h & 0x8000) ? -v : v;
}

// Smallest half-precision value >= x (x >= 0), as a float; +inf above 65504.
float half_round_up(double x) {
  if (!(x <= 65504.0)) return INFINITY;
  if (x <= 0.0) return 0.0f;
  int e;
  std::frexp(x, &e);  // x in [2^(e-1), 2^e)
  const double q = e - 1 < -14 ? std::ldexp(1.0, -24) : std::ldexp(1.0, e - 11);
  const double r = std::ceil(x / q) * q;
  return r > 65504.0 ? INFINITY : (float)r;
}

// Half-extents of the box around a splat's alpha >= 1/255 footprint.  Sec. 3.1
// skips a splat at a pixel where o G < 1/255, i.e. outside the ellipse
// d^T Q d <= tau with tau = 2 ln(255 o) and Q the conic [[A, B], [B, C]]; the box
// of that ellipse has half-widths sqrt(tau C / det Q) and sqrt(tau A / det Q).
// They are widened by 0.1% + 0.01 px and rounded up to half precision, the form
// in which the rasteriser keeps them; tau <= 0 gives -inf (no pixel reaches
// 1/255), a non-finite half-width +inf.  `s` scales tau and the ratios by
// (1 + s) (s < 0 shrinks): the rounding envelope of an FP32 evaluation.
void footprint_half_extents(double A, double B, double C, double o, double s, float& hx, float& hy) {
  const double tau0 = 2.0 * std::log(255.0 * o);
  const double tau = tau0 + s * (std::fabs(tau0) + 1.0);
  if (!(tau > 0.0)) {
    hx = hy = -INFINITY;
    return;
  }
  const double det = A * C - B * B;
  const double ex = std::sqrt(tau * C / det * (1.0 + s)), ey = std::sqrt(tau * A / det * (1.0 + s));
  if (!(ex < 1e30) || !(ey < 1e30)) {
    hx = hy = INFINITY;
    return;
  }
  hx = half_round_up(ex * 1.001 + 0.01);
  hy = half_round_up(ey * 1.001 + 0.01);
}

// Tile rectangle [x0, x1) x [y0, y1) of a splat, decided in FP32 from FP32 inputs.
// The 3DGS rule (Sec. 3.1) takes the tiles of the square of half-width r around
// the centre:
//   x0 = clamp(floor((mx - r) / tw), 0, Tx),  x1 = clamp(floor((mx + (r + tw - 1)) / tw), 0, Tx)
// (and the same for y); it is intersected with the tiles that the footprint box
// [mx - hx, mx + hx] x [my - hy, my + hy] reaches:
//   x0 >= floor((mx - hx) / tw),  x1 <= floor((mx + hx) / tw) + 1.
// A tile outside that box has no pixel where the splat is blended, so the
// intersection changes no image.  Each FP32 operation below rounds once.
void rect_f32(float mx, float my, int r, float hx, float hy, int tw, int th, int Tx, int Ty, int& x0, int& x1,
              int& y0, int& y1) {
  volatile float lo_x = mx - (float)r;
  volatile float hi_x = mx + (float)(r + tw - 1);
  volatile float lo_y = my - (float)r;
  volatile float hi_y = my + (float)(r + th - 1);
  volatile float flo_x = mx - hx, fhi_x = mx + hx;
  volatile float flo_y = my - hy, fhi_y = my + hy;
  float qx0 = lo_x / (float)tw, qx1 = hi_x / (float)tw;
  float qy0 = lo_y / (float)th, qy1 = hi_y / (float)th;
  float fx0 = flo_x / (float)tw, fx1 = fhi_x / (float)tw;
  float fy0 = flo_y / (float)th, fy1 = fhi_y / (float)th;
  auto cl = [](float f, int hi) {
    if (!(f > 0.0f)) return 0;  // also maps NaN to 0
    if (f > (float)hi) return hi;
    return (int)f;
  };
  x0 = std::max(cl(std::floor(qx0), Tx), cl(std::floor(fx0), Tx));
  x1 = std::min(cl(std::floor(qx1), Tx), cl(std::floor(fx1) + 1.0f, Tx));
  y0 = std::max(cl(std::floor(qy0), Ty), cl(std::floor(fy0), Ty));
  y1 = std::min(cl(std::floor(qy1), Ty), cl(std::floor(fy1) + 1.0f, Ty));
}

uint32_t f32_bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
}

// Per-row tiles of a splat within its rectangle (Sec. 3.1 skip rule, as for
// the box above): in units of the half-extents, u = dx/hx and v = dy/hy, the
// footprint ellipse d^T Q d <= tau reads u^2 - 2 rho u v + v^2 <= 1 - rho^2 with
// rho = -B / sqrt(A C) (hx^2 = tau C/det, hy^2 = tau A/det and the off-diagonal
// of tau Q^-1 is rho hx hy).  For a tile row, whose band is its full height
// [ty th, (ty + 1) th] in pixels, the ellipse's right end is
// rho v + sqrt((1 - rho^2)(1 - v^2)) at v = rho clamped into the band, the left
// end rho v - sqrt(...) at v = -rho clamped; both are widened by 1 % of hx +
// 0.5 px, and the row keeps the tiles from floor(left / tw) to floor(right / tw)
// within the rectangle.  A band outside |v| <= 1 keeps nothing.  Decided in
// FP32, one rounding per operation, in this order.  Without finite positive
// extents (or in the 3DGS-square mode) every row keeps the rectangle's row.
struct FootRowsF {
  float mx, my, hx, hy, rho, q, mgn;
  int x0, x1, y0, y1;
  bool exact;
};

FootRowsF foot_rows_f32(float mx, float my, float A, float B, float C, int r, float hx, float hy, bool footprint,
                        int tw, int th, int Tx, int Ty) {
  FootRowsF f;
  rect_f32(mx, my, r, footprint ? hx : INFINITY, footprint ? hy : INFINITY, tw, th, Tx, Ty, f.x0, f.x1, f.y0, f.y1);
  if (r <= 0) f.x1 = f.x0;
  f.mx = mx;
  f.my = my;
  f.hx = hx;
  f.hy = hy;
  f.exact = footprint && hx > 0.0f && hy > 0.0f && hx < 65536.0f && hy < 65536.0f && A > 0.0f && C > 0.0f;
  volatile float ac = A * C;
  volatile float sq = std::sqrt((float)ac);
  volatile float rho = -B / (float)sq;
  const float rc = std::fmin(std::fmax((float)rho, -1.0f), 1.0f);
  f.rho = f.exact ? rc : 0.0f;
  volatile float r2 = f.rho * f.rho;
  volatile float q = 1.0f - (float)r2;
  f.q = std::fmax(0.0f, (float)q);
  volatile float m1 = 0.01f * hx;
  volatile float m2 = (float)m1 + 0.5f;
  f.mgn = m2;
  return f;
}

int clamp_floor_f32(float f, int hi) {
  if (!(f > 0.0f)) return 0;  // also maps NaN to 0
  if (f > (float)hi) return hi;
  return (int)f;
}

// Tiles [a, b) of row ty.
void row_span_f32(const FootRowsF& f, int ty, int tw, int th, int Tx, int& a, int& b) {
  a = f.x0;
  b = f.x1;
  if (!f.exact) return;
  volatile float ylo = (float)(ty * th) - f.my;
  volatile float vlo = (float)ylo / f.hy;
  volatile float yhi = (float)((ty + 1) * th) - f.my;
  volatile float vhi = (float)yhi / f.hy;
  if ((float)vhi < -1.0f || (float)vlo > 1.0f) {
    b = a;
    return;
  }
  const float vr = std::fmin(std::fmax(f.rho, (float)vlo), (float)vhi);
  const float vl = std::fmin(std::fmax(-f.rho, (float)vlo), (float)vhi);
  volatile float vr2 = vr * vr;
  volatile float omr = 1.0f - (float)vr2;
  volatile float tr = f.q * (float)omr;
  volatile float sr = std::sqrt(std::fmax(0.0f, (float)tr));
  volatile float vl2 = vl * vl;
  volatile float oml = 1.0f - (float)vl2;
  volatile float tl = f.q * (float)oml;
  volatile float sl = std::sqrt(std::fmax(0.0f, (float)tl));
  volatile float pr = f.rho * vr;
  volatile float ur = (float)pr + (float)sr;
  volatile float hr = f.hx * (float)ur;
  volatile float xr0 = f.mx + (float)hr;
  volatile float xr = (float)xr0 + f.mgn;
  volatile float pl = f.rho * vl;
  volatile float ul = (float)pl - (float)sl;
  volatile float hl = f.hx * (float)ul;
  volatile float xl0 = f.mx + (float)hl;
  volatile float xl = (float)xl0 - f.mgn;
  volatile float qa = (float)xl / (float)tw;
  volatile float qb = (float)xr / (float)tw;
  a = std::max(a, clamp_floor_f32(std::floor((float)qa), Tx));
  b = std::min(b, clamp_floor_f32(std::floor((float)qb) + 1.0f, Tx));
  if (b < a) b = a;
}

struct Pair {
  uint64_t key;
  uint32_t val;
};

// All (tile, splat) pairs of all views, sorted by (key, splat index); key =
// (view * tiles_per_view + tile) << 32 | bits(depth).  `footprint`: the
// rectangle narrowed to the extents' box and row by row to the ellipse;
// otherwise the 3DGS square.
std::vector<Pair> bin_and_sort(int n_views, long n, const float* mx, const float* my, const float* A,
                               const float* B, const float* C, const int* rad, const float* hx, const float* hy,
                               const float* depth, int W, int H, int tw, int th, bool footprint) {
  int Tx = (W + tw - 1) / tw, Ty = (H + th - 1) / th;
  long T = (long)Tx * Ty;
  std::vector<Pair> pairs;
  for (int v = 0; v < n_views; ++v)
    for (long i = 0; i < n; ++i) {
      long gi = (long)v * n + i;
      if (rad[gi] <= 0) continue;
      const FootRowsF f =
          foot_rows_f32(mx[gi], my[gi], A[gi], B[gi], C[gi], rad[gi], hx[gi], hy[gi], footprint, tw, th, Tx, Ty);
      for (int ty = f.y0; ty < f.y1; ++ty) {
        int a, b;
        row_span_f32(f, ty, tw, th, Tx, a, b);
        for (int tx = a; tx < b; ++tx) {
          uint64_t tile = (uint64_t)v * T + (uint64_t)ty * Tx + tx;
          pairs.push_back({(tile << 32) | f32_bits(depth[gi]), (uint32_t)i});
        }
      }
    }
  std::sort(pairs.begin(), pairs.end(), [](const Pair& a, const Pair& b) {
    return a.key < b.key || (a.key == b.key && a.val < b.val);
  });
  return pairs;
}

// --------------------------------------------------------- per-view scene
struct View {
  Cam cam;
  int tw, th, Tx, Ty;
  std::vector<Splat<double>> sp;
  std::vector<std::vector<int>> lists;  // per tile, splat indices front to back
  // per splat, the tile rectangle when its FP32 inputs are moved to the edges of
  // their rounding uncertainty (lo shrinks, hi grows): x0, x1, y0, y1
  std::vector<int> lo, hi;
  // per tile, the splats that may enter or leave it under rounding
  std::vector<std::vector<int>> amb;
  // per splat: some tile of its own may enter or leave under rounding
  std::vector<char> own_amb;
  // per tile, for blend_flips: the splats of amb not in the list, in key order,
  // and the largest colour channel of the list's and those splats
  std::vector<std::vector<int>> amb_extra;
  std::vector<double> tile_cmax;
};

// Tiles whose membership in a splat's per-row spans may differ between the
// oracle's FP32 decision and the GPU's (their inputs differ by rounding): for
// every row of the grown rectangle, the tiles whose inclusion changes when the
// FP64 left or right end moves by delta (those just outside the end: the tile
// that holds the end is kept either way), and the whole row when its band is
// within rounding of |v| = 1.
// delta covers the half-precision step of hx (2^-10 relative), the error of rho
// from the FP32 conic (growing as 1 - rho^2 shrinks), the shift of the clamped
// v under the error of hy, and the centre's error.
void row_end_ambiguity(const Splat<double>& s, float hx, float hy, const int* hi_rect, int tw, int th,
                       std::vector<int>& tiles, int Tx) {
  if (!(hx > 0.0f && hy > 0.0f && hx < 65536.0f && hy < 65536.0f && s.A > 0.0 && s.C > 0.0)) return;
  const double rho = std::fmin(std::fmax(-s.B / std::sqrt(s.A * s.C), -1.0), 1.0);
  const double q = std::fmax(0.0, 1.0 - rho * rho);
  const double drho = 2e-6 / std::fmax(q, 1e-12) + 1e-6;
  const double mgn = 0.01 * hx + 0.5;
  // tiles [lo, hi] (clamped to the grown rectangle)
  auto add_tiles = [&](double lo, double hi, int ty) {
    const int a = std::max(hi_rect[0], (int)lo), b = std::min(hi_rect[1] - 1, (int)hi);
    for (int tx = a; tx <= b; ++tx) tiles.push_back(ty * Tx + tx);
  };
  const double dv1 = 1.5e-3 + 1e-5;  // rounding of v near |v| = 1
  for (int ty = hi_rect[2]; ty < hi_rect[3]; ++ty) {
    const double vlo = (ty * th - s.my) / hy, vhi = ((ty + 1) * th - s.my) / hy;
    if (vhi < -1.0 - dv1 || vlo > 1.0 + dv1) continue;
    if (std::fabs(vhi + 1.0) <= dv1 || std::fabs(vlo - 1.0) <= dv1) {
      for (int tx = hi_rect[0]; tx < hi_rect[1]; ++tx) tiles.push_back(ty * Tx + tx);
      continue;
    }
    for (int side = 0; side < 2; ++side) {
      const double sg = side == 0 ? 1.0 : -1.0;  // right end, then left end
      const double v = std::fmin(std::fmax(sg * rho, vlo), vhi);
      const double dv = 1.5e-3 * std::fabs(v) + 1e-5;
      const double root = std::sqrt(std::fmax(0.0, 1.0 - v * v));
      const double u = rho * v + sg * std::sqrt(q) * root;
      const double va = std::fmax(0.0, std::fabs(v) - dv);
      const double dsq = std::sqrt(std::fmax(0.0, 1.0 - va * va)) - root;
      const double d = hx * (1.5e-3 + drho * (1.0 + 1.0 / std::sqrt(std::fmax(q, 1e-12))) +
                             std::fabs(rho) * dv + std::sqrt(q) * dsq) +
                       1e-5 * (1.0 + std::fabs(s.mx)) + 1e-4;
      const double x = s.mx + hx * u + sg * mgn;
      if (side == 0)  // right end: tiles up to floor(x / tw) are kept
        add_tiles(std::floor((x - d) / tw) + 1, std::floor((x + d) / tw), ty);
      else  // left end: tiles from floor(x / tw) on are kept
        add_tiles(std::floor((x - d) / tw), std::floor((x + d) / tw) - 1, ty);
    }
  }
}

// Rounding envelopes of the FP32 inputs of a binning decision: the radius
// (3 sqrt(lambda_max) from a chain of FP32 products, ~1e-6 relative, widened
// 10x), the splat centre (a few FP32 ulps of its coordinate) and the footprint
// half-extents (tau and the conic ratios to 1e-4, plus the cancellation in the
// conic's determinant at FP32 precision).
const double kAmbRel = 1e-5;
const double kAmbCentreRel = 1e-6;
const double kAmbCentreAbs = 1e-5;
const double kAmbExtRel = 1e-4;

// Tiles of a splat in the renders: 0 its 3DGS square, 1 the square narrowed to
// its footprint box (set by or_set_footprint_bins).
int g_footprint_bins = 0;

View build_view(const double* P, long pitch, long n, int deg, const double* cam24, int tw, int th) {
  View V;
  V.cam = make_cam(cam24);
  V.tw = tw; V.th = th;
  V.Tx = (V.cam.W + tw - 1) / tw;
  V.Ty = (V.cam.H + th - 1) / th;
  V.sp.resize(n);
  std::vector<float> mx(n), my(n), dp(n), hx(n), hy(n), cA(n), cB(n), cC(n);
  std::vector<int> rad(n);
  V.lo.assign(4 * n, 0);
  V.hi.assign(4 * n, 0);
  V.own_amb.assign(n, 0);
  for (long i = 0; i < n; ++i) {
    G3<double> g = load_gaussian<double>(P, pitch, i, deg, nullptr);
    V.sp[i] = project(g, V.cam);
    const Splat<double>& s = V.sp[i];
    mx[i] = (float)s.mx; my[i] = (float)s.my; dp[i] = (float)s.depth;
    cA[i] = (float)s.A; cB[i] = (float)s.B; cC[i] = (float)s.C;
    rad[i] = s.valid ? s.radius : 0;
    if (!s.valid) continue;
    float hx_lo = INFINITY, hy_lo = INFINITY, hx_hi = INFINITY, hy_hi = INFINITY;
    hx[i] = hy[i] = INFINITY;
    if (g_footprint_bins) {
      footprint_half_extents(s.A, s.B, s.C, s.o, 0.0, hx[i], hy[i]);
      const double cancel = (s.A * s.C + s.B * s.B) / std::fabs(s.A * s.C - s.B * s.B);
      const double se = kAmbExtRel + 1e-6 * (std::isfinite(cancel) ? cancel : 1e30);
      footprint_half_extents(s.A, s.B, s.C, s.o, -se, hx_lo, hy_lo);
      footprint_half_extents(s.A, s.B, s.C, s.o, se, hx_hi, hy_hi);
    }
    double rr = s.radius_raw;
    int r_lo = (int)std::ceil(rr * (1.0 - kAmbRel) - 1e-6);
    int r_hi = (int)std::ceil(rr * (1.0 + kAmbRel) + 1e-6);
    double ex = kAmbCentreRel * (std::fabs(s.mx) + rr + tw) + kAmbCentreAbs;
    double ey = kAmbCentreRel * (std::fabs(s.my) + rr + th) + kAmbCentreAbs;
    int a0, a1, b0, b1, c0, c1, d0, d1;
    // shrunk rectangle: lower edges from the centre moved up, upper edges from it moved down
    rect_f32((float)(s.mx + ex), (float)(s.my + ey), r_lo, hx_lo, hy_lo, tw, th, V.Tx, V.Ty, a0, a1, b0, b1);
    rect_f32((float)(s.mx - ex), (float)(s.my - ey), r_lo, hx_lo, hy_lo, tw, th, V.Tx, V.Ty, c0, c1, d0, d1);
    V.lo[4 * i + 0] = a0; V.lo[4 * i + 1] = c1; V.lo[4 * i + 2] = b0; V.lo[4 * i + 3] = d1;
    rect_f32((float)(s.mx - ex), (float)(s.my - ey), r_hi, hx_hi, hy_hi, tw, th, V.Tx, V.Ty, a0, a1, b0, b1);
    rect_f32((float)(s.mx + ex), (float)(s.my + ey), r_hi, hx_hi, hy_hi, tw, th, V.Tx, V.Ty, c0, c1, d0, d1);
    V.hi[4 * i + 0] = a0; V.hi[4 * i + 1] = c1; V.hi[4 * i + 2] = b0; V.hi[4 * i + 3] = d1;
  }
  std::vector<Pair> pairs = bin_and_sort(1, n, mx.data(), my.data(), cA.data(), cB.data(), cC.data(), rad.data(),
                                         hx.data(), hy.data(), dp.data(), V.cam.W, V.cam.H, tw, th,
                                         g_footprint_bins != 0);
  V.lists.assign((size_t)V.Tx * V.Ty, {});
  for (const Pair& p : pairs) V.lists[p.key >> 32].push_back((int)p.val);
  V.amb.assign((size_t)V.Tx * V.Ty, {});
  std::vector<int> tiles;
  for (long i = 0; i < n; ++i) {
    if (!V.sp[i].valid) continue;
    const int* h = &V.hi[4 * i];
    const int* l = &V.lo[4 * i];
    tiles.clear();
    if (!(h[0] == l[0] && h[1] == l[1] && h[2] == l[2] && h[3] == l[3]))
      for (int ty = h[2]; ty < h[3]; ++ty)
        for (int tx = h[0]; tx < h[1]; ++tx)
          if (!(tx >= l[0] && tx < l[1] && ty >= l[2] && ty < l[3])) tiles.push_back(ty * V.Tx + tx);
    if (g_footprint_bins) row_end_ambiguity(V.sp[i], hx[i], hy[i], h, tw, th, tiles, V.Tx);
    if (tiles.empty()) continue;
    V.own_amb[i] = 1;
    std::sort(tiles.begin(), tiles.end());
    tiles.erase(std::unique(tiles.begin(), tiles.end()), tiles.end());
    for (int t : tiles) V.amb[(size_t)t].push_back((int)i);
  }
  V.amb_extra.assign((size_t)V.Tx * V.Ty, {});
  V.tile_cmax.assign((size_t)V.Tx * V.Ty, 0.0);
  auto cmax_of = [&](int i) { return std::max({V.sp[i].rgb[0], V.sp[i].rgb[1], V.sp[i].rgb[2], 0.0}); };
  for (size_t t = 0; t < V.lists.size(); ++t) {
    for (int i : V.lists[t]) V.tile_cmax[t] = std::max(V.tile_cmax[t], cmax_of(i));
    for (int i : V.amb[t])
      if (std::find(V.lists[t].begin(), V.lists[t].end(), i) == V.lists[t].end()) {
        V.amb_extra[t].push_back(i);
        V.tile_cmax[t] = std::max(V.tile_cmax[t], cmax_of(i));
      }
    std::sort(V.amb_extra[t].begin(), V.amb_extra[t].end(), [&](int a, int b) {
      const float da = (float)V.sp[a].depth, db = (float)V.sp[b].depth;
      return da < db || (da == db && a < b);
    });
  }
  return V;
}

// --------------------------------------------------------------- blending
struct Contrib {
  int i;          // splat index
  double alpha;   // min(0.99, o G)
  double G;       // exp(power)
  bool capped;    // o G > 0.99
  double T;       // transmittance in front of this splat
  double dx, dy;  // mean - pixel centre
};

const double kAlphaMin = 1.0 / 255.0;
const double kAlphaMax = 0.99;
const double kTMin = 1e-4;

// Front-to-back blend of one pixel (Sec. 3.1): skip a splat whose power is
// positive or whose alpha is below 1/255, stop before the splat that would bring
// T below 1e-4, black background.  n_contrib = 1 + list position of the last
// splat blended.  `margin` receives the smallest relative distance of any
// decision taken to its threshold.
template <class S>
void blend(const std::vector<int>& list, const std::vector<Splat<S>>& sp, double pcx, double pcy,
           S C[3], S& T, int& n_contrib, double* margin, std::vector<Contrib>* trace) {
  T = S(1.0);
  C[0] = C[1] = C[2] = S(0.0);
  n_contrib = 0;
  double mg = std::numeric_limits<double>::infinity();
  for (size_t k = 0; k < list.size(); ++k) {
    const Splat<S>& g = sp[list[k]];
    S dx = g.mx - S(pcx), dy = g.my - S(pcy);
    S power = -0.5 * (g.A * dx * dx + g.C * dy * dy) - g.B * dx * dy;
    mg = std::min(mg, std::fabs(val(power)) * 1e6);
    if (val(power) > 0.0) continue;
    S G = exp(power);
    S oG = g.o * G;
    bool capped = val(oG) > kAlphaMax;
    mg = std::min(mg, std::fabs(val(oG) - kAlphaMax) / kAlphaMax);
    S alpha = capped ? S(kAlphaMax) : oG;
    mg = std::min(mg, std::fabs(val(alpha) - kAlphaMin) / kAlphaMin);
    if (val(alpha) < kAlphaMin) continue;
    S Tn = T * (1.0 - alpha);
    mg = std::min(mg, std::fabs(val(Tn) - kTMin) / kTMin);
    if (val(Tn) < kTMin) break;
    if (trace) trace->push_back({list[k], val(alpha), val(G), capped, val(T), val(dx), val(dy)});
    for (int ch = 0; ch < 3; ++ch) C[ch] = C[ch] + g.rgb[ch] * alpha * T;
    T = Tn;
    n_contrib = (int)k + 1;
  }
  if (margin) *margin = mg;
}

// 0 for pixels whose value may legitimately differ between an FP32 and an FP64
// evaluation because a splat's tile set, or the depth order of two splats, lies
// within rounding of a boundary; +inf otherwise.  `nc` is the pixel's n_contrib:
// a splat whose tile membership is ambiguous moves the list position of every
// later splat, so it also makes n_contrib ambiguous when it sorts before the
// pixel's last blended splat.  If it is not visible at the pixel (alpha below
// half the skip threshold, so skipped on both sides) only n_contrib moves: with
// nc_lo / nc_hi given, the range of n_contrib that the possible tile sets give
// is written there ([nc - ambiguous splats in the list before it, nc + those not
// in the list]) and the pixel is kept; without them it is excluded.
double binning_margin(const View& V, int tx, int ty, double pcx, double pcy, int nc = 0, int* nc_lo = nullptr,
                      int* nc_hi = nullptr) {
  const std::vector<int>& list = V.lists[(size_t)ty * V.Tx + tx];
  auto visible_at = [&](long i) {
    const Splat<double>& g = V.sp[i];
    double dx = g.mx - pcx, dy = g.my - pcy;
    double power = -0.5 * (g.A * dx * dx + g.C * dy * dy) - g.B * dx * dy;
    return g.o * std::exp(power) >= 0.5 * kAlphaMin;
  };
  auto before_last = [&](long i) {
    if (nc <= 0) return false;
    const long j = list[nc - 1];
    const float di = (float)V.sp[i].depth, dj = (float)V.sp[j].depth;
    return di < dj || (di == dj && i <= j);
  };
  int in_list = 0, off_list = 0;
  for (int i : V.amb[(size_t)ty * V.Tx + tx]) {
    if (visible_at(i)) return 0.0;
    if (!before_last(i)) continue;
    if (!nc_lo) return 0.0;
    if (std::find(list.begin(), list.end(), i) != list.end())
      ++in_list;
    else
      ++off_list;
  }
  if (nc_lo) {
    *nc_lo = nc - in_list;
    *nc_hi = nc + off_list;
  }
  for (size_t k = 1; k < list.size(); ++k) {
    double d0 = V.sp[list[k - 1]].depth, d1 = V.sp[list[k]].depth;
    if (std::fabs(d1 - d0) <= 1e-6 * std::fabs(d1) && visible_at(list[k - 1]) && visible_at(list[k]))
      return 0.0;
  }
  return std::numeric_limits<double>::infinity();
}

// Cotangents of the 2-D splat quantities, 9 per splat: (mx, my, A, B, C, o, r, g, b).
enum { Q_MX, Q_MY, Q_A, Q_B, Q_C, Q_O, Q_R, Q_G, Q_BL, NQ };

// ------------------------------------------------ FP32 decision uncertainty
// The CUDA path takes the blend's discrete decisions (Sec. 3.1 thresholds) on
// FP32 splat records, which differ from the oracle's FP64 ones by rounding.  A
// decision whose FP64 value lies closer to its threshold than that rounding can
// move it may come out the other way there.  The model below bounds the
// rounding: the record's mean carries a few ulps of its pixel coordinates
// (camera transform, perspective division and principal point, each rounded in
// FP32), its conic a few ulps relative to its entries, amplified by 1/(1 - rho^2)
// when the inversion cancels (rho the conic's correlation), and exp and the
// opacity a few ulps.  Returns the bound on |power_FP32 - power_FP64| at offset
// (dx, dy) from the mean.
double power_uncertainty(const Splat<double>& g, double dx, double dy) {
  const double ulp = std::ldexp(1.0, -24);
  const double dpos = 4.0 * ulp * (std::fabs(g.mx) + std::fabs(g.my)) + 1e-6;  // pixels
  const double rho2 = std::min(g.B * g.B / std::max(g.A * g.C, 1e-300), 0.999999);
  const double dconic = 32.0 * ulp / (1.0 - rho2);                               // relative
  const double gx = std::fabs(g.A * dx + g.B * dy), gy = std::fabs(g.B * dx + g.C * dy);
  const double q = 0.5 * (std::fabs(g.A) * dx * dx + std::fabs(g.C) * dy * dy) + std::fabs(g.B * dx * dy);
  return (gx + gy) * dpos + q * dconic + 1e-6;
}

// Where FP32 may flip the blend's decisions at one pixel, and what that can do.
//   impact    bound on |C_FP32 - C_FP64| from decisions that may flip (per
//             channel, the largest): dropping or adding a splat k moves the
//             colour by at most a_k T_k (c_k + c_max) (its own term plus the
//             (1 - a_k) it puts on everything behind it, whose colours sum to at
//             most T_k c_max); an earlier or later termination at k moves it by
//             at most T_k c_max; swapping two splats of nearly equal depth by
//             T a_i a_j c_max.
//   t_impact  the same bound for the final transmittance.
//   nc_lo, nc_hi  the n_contrib values those flips allow.
//   err       bound on the rounding of the colour itself with every decision
//             as here: sum over blended splats of c_k a_k T_k times the relative
//             rounding of a_k (from power_uncertainty) and of T_k (accumulated).
// Decisions whose FP64 value is farther from the threshold than the rounding
// bound (power_uncertainty, and for the termination test the transmittance's
// own accumulated rounding plus the changes upstream flips make to it) are
// firm.  The tile's amb splats (see build_view) are those whose membership in
// its list may differ: those in the list may be missing on the GPU, the others
// (amb_extra) may be present there.
// A decision of splat i's own at one pixel that FP32 may flip (its 1/255 skip,
// its cap, its power sign) or its membership in the tile's list: its alpha with
// the cap lifted, exp(power), offset from the pixel and the transmittance in
// front of it.
struct OwnFlip {
  int i;
  double a, G, dx, dy, T;
};

// The terms splat g adds at one pixel for the cotangent w, as absolute values,
// with its alpha uncapped: a bound on how far its reverse-pass terms there move
// when a decision of its own flips (added, dropped or uncapped).  cmax bounds
// the colours behind it (the suffix over 1 - a is at most T cmax / (1 - a)).
void own_terms(const Splat<double>& g, const OwnFlip& q, double cmax, const double w[3], double* out) {
  double gab = 0.0;
  for (int ch = 0; ch < 3; ++ch) gab += std::fabs(w[ch]) * q.T * (std::fabs(g.rgb[ch]) + cmax / (1.0 - q.a));
  out[Q_R] += std::fabs(w[0]) * q.a * q.T;
  out[Q_G] += std::fabs(w[1]) * q.a * q.T;
  out[Q_BL] += std::fabs(w[2]) * q.a * q.T;
  out[Q_O] += gab * q.G;
  const double gpow = gab * q.a;
  out[Q_A] += 0.5 * q.dx * q.dx * gpow;
  out[Q_B] += std::fabs(q.dx * q.dy) * gpow;
  out[Q_C] += 0.5 * q.dy * q.dy * gpow;
  out[Q_MX] += (std::fabs(g.A * q.dx) + std::fabs(g.B * q.dy)) * gpow;
  out[Q_MY] += (std::fabs(g.C * q.dy) + std::fabs(g.B * q.dx)) * gpow;
}

struct Flip {
  double impact = 0.0, t_impact = 0.0, err = 0.0;
  int nc_lo = 0, nc_hi = 0;
  int kinds = 0;  // flips that count: 1 skip, 2 termination, 4 list membership, 8 depth order
};

// owns (may be null) receives the splats whose own decision (skip, cap or
// power sign) or list membership may flip here, in walk order.
Flip blend_flips(const View& V, size_t tile, double pcx, double pcy, int nc, std::vector<OwnFlip>* owns = nullptr) {
  const std::vector<int>& list = V.lists[tile];
  const std::vector<int>& maybe = V.amb[tile];
  const std::vector<int>& extra = V.amb_extra[tile];
  const std::vector<Splat<double>>& sp = V.sp;
  Flip f;
  f.nc_lo = f.nc_hi = nc;
  struct Entry {
    int i;
    bool in_list;
    float depth;
  };
  auto cmax_of = [&](int i) { return std::max({sp[i].rgb[0], sp[i].rgb[1], sp[i].rgb[2], 0.0}); };
  const double cmax = V.tile_cmax[tile];
  auto is_maybe = [&](int i) { return std::find(maybe.begin(), maybe.end(), i) != maybe.end(); };
  double T = 1.0;
  double rho = 0.0;  // relative change of T that upstream flips can make
  double tun = 0.0;  // relative rounding of T accumulated by the FP32 products
  int pos = 0, firm_last = 0, maybe_before = 0;
  std::vector<int> extra_at;  // list positions at which possibly-present splats sort
  double prev_depth = -1.0, prev_a = 0.0;
  int prev_i = -1;
  bool drop_rest = false;  // a termination the GPU may take earlier lies in front
  bool prev_blended = false;
  // the walk order: the list, with the possibly-present splats merged in by key
  size_t li = 0, ei = 0;
  while (li < list.size() || ei < extra.size()) {
    Entry e;
    if (ei < extra.size()) {
      const int a = extra[ei];
      const float da = (float)sp[a].depth;
      bool take = li == list.size();
      if (!take) {
        const float dl = (float)sp[list[li]].depth;
        take = da < dl || (da == dl && a < list[li]);
      }
      if (take) {
        e = {a, false, da};
        ++ei;
      } else {
        e = {list[li], true, (float)sp[list[li]].depth};
        ++li;
      }
    } else {
      e = {list[li], true, (float)sp[list[li]].depth};
      ++li;
    }
    const Splat<double>& g = sp[e.i];
    const double dx = g.mx - pcx, dy = g.my - pcy;
    const double power = -0.5 * (g.A * dx * dx + g.C * dy * dy) - g.B * dx * dy;
    const double dp = power_uncertainty(g, dx, dy);
    const double oG = g.o * std::exp(std::min(power, 0.0));
    const bool capped = oG > kAlphaMax;
    const double a = capped ? kAlphaMax : oG;
    const bool blends = power <= 0.0 && a >= kAlphaMin;
    const bool near = std::fabs(power) <= dp || (!capped && std::fabs(a / kAlphaMin - 1.0) <= dp + 2e-6);
    const double drop = a * T * (cmax_of(e.i) + cmax);  // colour bound of adding or dropping it
    if (owns && oG >= 0.5 * kAlphaMin &&
        (near || !e.in_list || is_maybe(e.i) || std::fabs(oG / kAlphaMax - 1.0) <= dp + 2e-6))
      owns->push_back({e.i, std::min(oG, 1.0 - 1e-6), oG / g.o, dx, dy, T});
    if (!e.in_list) {
      // may be listed on the GPU: an extra splat wherever it would blend
      if (blends || near) {
        f.kinds |= 4;
        f.impact += drop;
        f.t_impact += a * T;
        rho += a / (1.0 - a);
      }
      extra_at.push_back(pos);
      continue;
    }
    const int k = pos++;
    if (k < nc && is_maybe(e.i)) ++maybe_before;  // may be missing on the GPU: later positions move up
    if (!blends) {
      if (near) {  // skipped here, may blend on the GPU
        f.kinds |= 1;
        f.impact += drop;
        f.t_impact += a * T;
        rho += a / (1.0 - a);
        f.nc_hi = std::max(f.nc_hi, k + 1);
      }
      continue;
    }
    // blended here; the termination test first
    const double Tn = T * (1.0 - a);
    const double da = capped ? 0.0 : (dp + 2e-6) * a / (1.0 - a);
    const bool near_term = std::fabs(Tn / kTMin - 1.0) <= tun + rho + da + 1e-6;
    if (Tn < kTMin) {
      if (near_term) {  // the GPU may go on past this point
        f.kinds |= 2;
        f.impact += T * cmax;
        f.t_impact += T;
        f.nc_hi = (int)list.size();
        if (owns) {
          // the splats it may then blend, from this one on, at most at this T
          double Tc = T;
          const size_t from = li - 1;  // this splat's list index
          for (size_t u = from; u < list.size() && Tc >= 0.5 * kTMin; ++u) {
            const Splat<double>& h = sp[list[u]];
            const double hx = h.mx - pcx, hy = h.my - pcy;
            const double hp = -0.5 * (h.A * hx * hx + h.C * hy * hy) - h.B * hx * hy;
            const double hoG = h.o * std::exp(std::min(hp, 0.0));
            if (hoG < 0.5 * kAlphaMin) continue;
            const double ha = std::min(hoG, 1.0 - 1e-6);
            owns->push_back({list[u], ha, hoG / h.o, hx, hy, Tc});
            Tc *= 1.0 - std::min(hoG, kAlphaMax);
          }
        }
      }
      break;
    }
    if (near_term) {  // the GPU may stop here: this splat and all behind it may be missing
      f.kinds |= 2;
      f.impact += T * cmax;
      f.t_impact += T;
      f.nc_lo = std::min(f.nc_lo, firm_last);
      drop_rest = true;
    }
    if (owns && drop_rest && !(near || !e.in_list || is_maybe(e.i) || std::fabs(oG / kAlphaMax - 1.0) <= dp + 2e-6))
      owns->push_back({e.i, std::min(oG, 1.0 - 1e-6), oG / g.o, dx, dy, T});
    const bool amb = is_maybe(e.i);
    if (near || amb) {
      f.kinds |= near ? 1 : 4;
      f.impact += drop;
      f.t_impact += a * T;
      rho += a / (1.0 - a);
    } else {
      firm_last = k + 1;
    }
    // two consecutive blended splats whose FP32 depths (a few ulps apart on the
    // two sides) may sort the other way: the swap moves the colour by
    // T a_i a_j (c_i - c_j), T the transmittance in front of the pair
    if (prev_blended && std::fabs((double)e.depth - prev_depth) <= 4.0 * std::ldexp(std::fabs(prev_depth), -23)) {
      double dc = 0.0;
      for (int ch = 0; ch < 3; ++ch) dc = std::max(dc, std::fabs(g.rgb[ch] - sp[prev_i].rgb[ch]));
      f.kinds |= 8;
      f.impact += T / (1.0 - prev_a) * prev_a * a * dc;
    }
    prev_blended = true;
    prev_depth = e.depth;
    prev_a = a;
    prev_i = e.i;
    f.err += cmax_of(e.i) * a * T * ((capped ? 0.0 : dp + 2e-6) + tun + 2e-7);
    tun += (capped ? 0.0 : (dp + 2e-6) * a / (1.0 - a)) + 2e-7;
    T = Tn;
  }
  f.nc_lo = std::min(f.nc_lo, firm_last) - maybe_before;
  int extra_before = 0;  // possibly-present splats in front of the last possible contributor
  for (int at : extra_at) extra_before += at < f.nc_hi;
  f.nc_hi += extra_before;
  return f;
}

// The tolerance the CUDA path's images are held to (max-abs): residuals of the
// two sides differ by at most this where the images are compared.
// Every result of the blend at one pixel that an FP32 evaluation may reach, as
// the sequences of splats blended, front to back.  The walk takes the tile's
// list with the possibly-present splats merged in by key (as blend_flips) and
// takes every decision as FP64 does, except that each decision blend_flips
// counts as possibly flipped is taken both ways: a splat that may be skipped or
// blended (its 1/255 skip or its power sign within the rounding bound of
// power_uncertainty, or its membership in the tile's list ambiguous), a
// termination within the transmittance's rounding of 1e-4, and the order of two
// splats that may blend whose FP32 depths are a few ulps apart.  A flip whose
// bound on the colour and on T (as in blend_flips) is at most branch_min is not
// taken both ways: its bound is summed along the path instead, and its relative
// change of T widens later termination tests.  The FP64 walk's own sequence is
// the last leaf.  rest / t_rest receive the largest sums over the leaves.
// Returns false (leaves incomplete) when there would be more than max_leaves.
struct BlendOutcomes {
  const View& V;
  double pcx, pcy, cmax, branch_min;
  size_t max_leaves;
  struct Entry {
    int i;
    bool in_list, maybe;
    float depth;
  };
  std::vector<Entry> E;
  std::vector<std::vector<int>> leaves;
  double rest = 0.0, t_rest = 0.0;
  bool overflow = false;

  BlendOutcomes(const View& V_, size_t tile, double x, double y, double bmin, size_t maxl)
      : V(V_), pcx(x), pcy(y), cmax(V_.tile_cmax[tile]), branch_min(bmin), max_leaves(maxl) {
    const std::vector<int>& list = V.lists[tile];
    const std::vector<int>& maybe = V.amb[tile];
    const std::vector<int>& extra = V.amb_extra[tile];
    size_t li = 0, ei = 0;
    while (li < list.size() || ei < extra.size()) {
      bool take_extra = ei < extra.size();
      if (take_extra && li < list.size()) {
        const float da = (float)V.sp[extra[ei]].depth, dl = (float)V.sp[list[li]].depth;
        take_extra = da < dl || (da == dl && extra[ei] < list[li]);
      }
      const int i = take_extra ? extra[ei++] : list[li++];
      const bool amb = !take_extra && std::find(maybe.begin(), maybe.end(), i) != maybe.end();
      E.push_back({i, !take_extra, amb, (float)V.sp[i].depth});
    }
  }

  struct Eval {
    double a, dp, drop;
    bool capped, blends, near;
  };
  Eval eval(int i, double T) const {
    const Splat<double>& g = V.sp[i];
    const double dx = g.mx - pcx, dy = g.my - pcy;
    const double power = -0.5 * (g.A * dx * dx + g.C * dy * dy) - g.B * dx * dy;
    Eval r;
    r.dp = power_uncertainty(g, dx, dy);
    const double oG = g.o * std::exp(std::min(power, 0.0));
    r.capped = oG > kAlphaMax;
    r.a = r.capped ? kAlphaMax : oG;
    r.blends = power <= 0.0 && r.a >= kAlphaMin;
    r.near = std::fabs(power) <= r.dp || (!r.capped && std::fabs(r.a / kAlphaMin - 1.0) <= r.dp + 2e-6);
    const double ci = std::max({g.rgb[0], g.rgb[1], g.rgb[2], 0.0});
    r.drop = r.a * T * (ci + cmax);
    return r;
  }
  // may the splat blend at this pixel on either side
  static bool may_blend(const Eval& r) { return r.blends || r.near; }

  void leaf(const std::vector<int>& seq, double rs, double trs) {
    if (leaves.size() >= max_leaves) {
      overflow = true;
      return;
    }
    leaves.push_back(seq);
    rest = std::max(rest, rs);
    t_rest = std::max(t_rest, trs);
  }

  // From entry p on, with transmittance T, its accumulated relative rounding
  // tun, the relative change rho that unbranched flips may make to it, and the
  // sums of unbranched bounds rs / trs.  no_swap: entry p is the later splat of a
  // pair already swapped.
  void walk(size_t p, std::vector<int> seq, double T, double tun, double rho, double rs, double trs, bool no_swap) {
    for (; p < E.size() && !overflow; ++p, no_swap = false) {
      Eval r = eval(E[p].i, T);
      if (!no_swap && may_blend(r)) {
        // the next splat that may blend: if its depth is within a few ulps, the
        // GPU's keys may put it first
        size_t q = p + 1;
        Eval rq{};
        for (; q < E.size(); ++q) {
          rq = eval(E[q].i, T);
          if (may_blend(rq)) break;
        }
        const double d0 = E[p].depth;
        if (q < E.size() && std::fabs((double)E[q].depth - d0) <= 4.0 * std::ldexp(std::fabs(d0), -23)) {
          double dc = 0.0;
          for (int ch = 0; ch < 3; ++ch) dc = std::max(dc, std::fabs(V.sp[E[p].i].rgb[ch] - V.sp[E[q].i].rgb[ch]));
          const double sw = T * r.a * rq.a * dc;
          if (sw > branch_min) {
            std::swap(E[p], E[q]);
            walk(p, seq, T, tun, rho, rs, trs, true);
            std::swap(E[p], E[q]);
            if (overflow) return;
          } else {
            rs += sw;
          }
        }
      }
      const Entry& e = E[p];
      const bool fp64_blend = e.in_list && r.blends;
      const bool alt = fp64_blend ? (r.near || e.maybe) : (e.in_list ? r.near : (r.blends || r.near));
      const bool small = r.drop <= branch_min && r.a * T <= branch_min;
      if (alt && small) {  // summed, not taken both ways
        rs += r.drop;
        trs += r.a * T;
        rho += r.a / (1.0 - r.a);
      }
      const bool try_blend = fp64_blend || (alt && !small);
      const bool try_skip = !fp64_blend || (alt && !small);
      if (try_blend) {
        const double Tn = T * (1.0 - r.a);
        const double da = r.capped ? 0.0 : (r.dp + 2e-6) * r.a / (1.0 - r.a);
        const bool near_term = std::fabs(Tn / kTMin - 1.0) <= tun + rho + da + 1e-6;
        const bool stop64 = Tn < kTMin;
        const bool term_small = T * cmax <= branch_min && T <= branch_min;
        if (near_term && term_small) {
          rs += T * cmax;
          trs += T;
        }
        const bool both = near_term && !term_small;
        const double tun_n = tun + (r.capped ? 0.0 : (r.dp + 2e-6) * r.a / (1.0 - r.a)) + 2e-7;
        // the outcomes of blending it: stop in front of it, or blend and go on
        const bool may_stop = stop64 || both, may_go = !stop64 || both;
        if (fp64_blend) {
          // the FP64 outcome is followed in this loop; the others first
          if (try_skip) walk(p + 1, seq, T, tun, rho, rs, trs, false);
          if (stop64) {
            if (may_go) {
              std::vector<int> s2 = seq;
              s2.push_back(e.i);
              walk(p + 1, s2, Tn, tun_n, rho, rs, trs, false);
            }
            leaf(seq, rs, trs);
            return;
          }
          if (may_stop) leaf(seq, rs, trs);
          seq.push_back(e.i);
          T = Tn;
          tun = tun_n;
          continue;
        }
        // FP64 skips it: the blended alternatives first
        if (may_stop) leaf(seq, rs, trs);
        if (may_go) {
          std::vector<int> s2 = seq;
          s2.push_back(e.i);
          walk(p + 1, s2, Tn, tun_n, rho, rs, trs, false);
        }
      }
      // skipped (FP64's outcome when it does not blend)
    }
    if (!overflow) leaf(seq, rs, trs);
  }
};

// The blend of one pixel over a given sequence of splats (every one blended, in
// order): C = sum_k c_k a_k T_k with a_k = min(0.99, o_k G_k) (Sec. 3.1).  get(i)
// returns splat i.
template <class S, class Get>
void blend_sequence(const std::vector<int>& seq, Get get, double pcx, double pcy, S C[3], S& T) {
  T = S(1.0);
  C[0] = C[1] = C[2] = S(0.0);
  for (int i : seq) {
    const Splat<S>& g = get(i);
    S dx = g.mx - S(pcx), dy = g.my - S(pcy);
    S power = -0.5 * (g.A * dx * dx + g.C * dy * dy) - g.B * dx * dy;
    S oG = g.o * exp(power);
    S alpha = val(oG) > kAlphaMax ? S(kAlphaMax) : oG;
    for (int ch = 0; ch < 3; ++ch) C[ch] = C[ch] + g.rgb[ch] * alpha * T;
    T = T * (1.0 - alpha);
  }
}

const double kImageTol = 1e-5;

// Calls f(tx, ty, x, y) for every pixel of the view, tile by tile.
template <class F>
void for_each_pixel(const View& V, F f) {
  for (int ty = 0; ty < V.Ty; ++ty)
    for (int tx = 0; tx < V.Tx; ++tx)
      for (int y = ty * V.th; y < std::min((ty + 1) * V.th, V.cam.H); ++y)
        for (int x = tx * V.tw; x < std::min((tx + 1) * V.tw, V.cam.W); ++x) f(tx, ty, x, y);
}

// ------------------------------------------------------------ Rademacher
const uint64_t kGolden = 0x9E3779B97F4A7C15ULL;

// SplitMix64 output for state x (Steele, Lea & Flood 2014): one Weyl increment,
// then the finaliser with shifts 30, 27, 31.
uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + kGolden;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Entry j of Rademacher probe k at step t (the paper leaves the generator open):
// bit j mod 64 of the hash of word j / 64, so one hash gives 64 entries; a set
// bit is -1.
double rademacher(uint64_t seed, int64_t t, int k, uint64_t j) {
  uint64_t h = splitmix64(seed ^ ((uint64_t)t * kGolden) ^ ((uint64_t)k << 56) ^ (j >> 6));
  return ((h >> (j & 63)) & 1ULL) ? -1.0 : 1.0;
}

// Probe entry of parameter row r of Gaussian i: the rows of one Gaussian are
// consecutive entries, so they share one or two hashes.
uint64_t probe_entry(long i, int r, int rows) { return (uint64_t)i * (uint64_t)rows + (uint64_t)r; }

// ------------------------------------------------------------------ SSIM
// Per-pixel structural similarity of one channel x (rendered) against y
// (target), H x W row-major: local statistics under the 11 x 11 Gaussian window
// of standard deviation 1.5 (normalised over the whole window; pixels outside
// the image count as 0), C1 = 0.01^2, C2 = 0.03^2:
//   S = (2 mx my + C1)(2 sxy + C2) / ((mx^2 + my^2 + C1)(sx2 + sy2 + C2))
// with mx = G*x, sx2 = G*(x^2) - mx^2, sxy = G*(xy) - mx my.  As a function of
// the filtered raw moments (mx, Ex2 = G*(x^2), Exy = G*(xy)) its partials are
//   dS/dmx  = 2 A2/(B1 B2) (my - mx A1/B1) + 2 mx A1 A2/(B1 B2^2) - 2 my A1/(B1 B2)
//   dS/dEx2 = -A1 A2/(B1 B2^2),   dS/dExy = 2 A1/(B1 B2)
// (A1 = 2 mx my + C1, A2 = 2 sxy + C2, B1 = mx^2 + my^2 + C1, B2 = sx2 + sy2 + C2).
const int kSsimR = 5;
const double kSsimC1 = 1e-4, kSsimC2 = 9e-4;

std::vector<double> ssim_window() {
  std::vector<double> g(2 * kSsimR + 1);
  double s = 0.0;
  for (int i = -kSsimR; i <= kSsimR; ++i) s += g[i + kSsimR] = std::exp(-(double)(i * i) / (2.0 * 1.5 * 1.5));
  for (double& v : g) v /= s;
  return g;
}

// G * f at every pixel (zero outside the image), by direct window sums.
std::vector<double> ssim_filter(const double* f, int H, int W) {
  const std::vector<double> g = ssim_window();
  std::vector<double> out((size_t)H * W, 0.0);
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      double acc = 0.0;
      for (int dy = -kSsimR; dy <= kSsimR; ++dy)
        for (int dx = -kSsimR; dx <= kSsimR; ++dx) {
          int yy = y + dy, xx = x + dx;
          if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
          acc += g[dy + kSsimR] * g[dx + kSsimR] * f[(size_t)yy * W + xx];
        }
      out[(size_t)y * W + x] = acc;
    }
  return out;
}

struct SsimMaps {
  std::vector<double> S, dmx, dex2, dexy;
};

SsimMaps ssim_maps(const double* x, const double* y, int H, int W) {
  const size_t N = (size_t)H * W;
  std::vector<double> x2(N), y2(N), xy(N);
  for (size_t i = 0; i < N; ++i) {
    x2[i] = x[i] * x[i];
    y2[i] = y[i] * y[i];
    xy[i] = x[i] * y[i];
  }
  std::vector<double> mx = ssim_filter(x, H, W), my = ssim_filter(y, H, W);
  std::vector<double> ex2 = ssim_filter(x2.data(), H, W), ey2 = ssim_filter(y2.data(), H, W);
  std::vector<double> exy = ssim_filter(xy.data(), H, W);
  SsimMaps M;
  M.S.resize(N);
  M.dmx.resize(N);
  M.dex2.resize(N);
  M.dexy.resize(N);
  for (size_t i = 0; i < N; ++i) {
    const double sx2 = ex2[i] - mx[i] * mx[i], sy2 = ey2[i] - my[i] * my[i], sxy = exy[i] - mx[i] * my[i];
    const double A1 = 2 * mx[i] * my[i] + kSsimC1, A2 = 2 * sxy + kSsimC2;
    const double B1 = mx[i] * mx[i] + my[i] * my[i] + kSsimC1, B2 = sx2 + sy2 + kSsimC2;
    M.S[i] = A1 * A2 / (B1 * B2);
    // partials with respect to mx, sx2, sxy, then to the raw moments
    const double d_mx = 2 * A2 / (B1 * B2) * (my[i] - mx[i] * A1 / B1);
    const double d_sx2 = -A1 * A2 / (B1 * B2 * B2);
    const double d_sxy = 2 * A1 / (B1 * B2);
    M.dmx[i] = d_mx - 2 * mx[i] * d_sx2 - my[i] * d_sxy;
    M.dex2[i] = d_sx2;
    M.dexy[i] = d_sxy;
  }
  return M;
}

// sum_p a_p dS_p/dx_q for every q (the adjoint of the map x -> S).
std::vector<double> ssim_vjp(const double* x, const double* y, int H, int W, const SsimMaps& M, const double* a) {
  const size_t N = (size_t)H * W;
  std::vector<double> p1(N), p2(N), p3(N);
  for (size_t i = 0; i < N; ++i) {
    p1[i] = a[i] * M.dmx[i];
    p2[i] = a[i] * M.dex2[i];
    p3[i] = a[i] * M.dexy[i];
  }
  // the window is symmetric, so the adjoint filter is the filter itself
  std::vector<double> f1 = ssim_filter(p1.data(), H, W), f2 = ssim_filter(p2.data(), H, W);
  std::vector<double> f3 = ssim_filter(p3.data(), H, W);
  std::vector<double> out(N);
  for (size_t q = 0; q < N; ++q) out[q] = f1[q] + 2 * x[q] * f2[q] + y[q] * f3[q];
  return out;
}

// The directional derivative of S along the image direction d.
std::vector<double> ssim_jvp(const double* x, const double* y, int H, int W, const SsimMaps& M, const double* d) {
  const size_t N = (size_t)H * W;
  std::vector<double> xd(N), yd(N);
  for (size_t i = 0; i < N; ++i) {
    xd[i] = 2 * x[i] * d[i];
    yd[i] = y[i] * d[i];
  }
  std::vector<double> f1 = ssim_filter(d, H, W), f2 = ssim_filter(xd.data(), H, W), f3 = ssim_filter(yd.data(), H, W);
  std::vector<double> out(N);
  for (size_t i = 0; i < N; ++i) out[i] = M.dmx[i] * f1[i] + M.dex2[i] * f2[i] + M.dexy[i] * f3[i];
  return out;
}

// ----------------------------------------------------------- reverse pass
// Cotangents of the 2-D splat quantities, 9 per splat (the enum Q_* above).

// Reverse pass of one pixel's blend, written out from
//   dC/dc_i = a_i T_i,
//   dC/da_i = c_i T_i - (sum_{j>i} c_j a_j T_j) / (1 - a_i),
//   a = o exp(power) (no derivative where a is capped at 0.99),
//   power = -1/2 (A dx^2 + C dy^2) - B dx dy with dx = mx - px, dy = my - py.
// `w` is dL/dC at the pixel; the result is added to cot[i * NQ + q].
void blend_reverse(const std::vector<Contrib>& tr, const std::vector<Splat<double>>& sp,
                   const double w[3], double* cot) {
  // suffix[k] = sum over later splats j of c_j a_j T_j
  std::vector<double> suffix(3 * (tr.size() + 1), 0.0);
  for (long k = (long)tr.size() - 1; k >= 0; --k)
    for (int ch = 0; ch < 3; ++ch)
      suffix[3 * k + ch] = suffix[3 * (k + 1) + ch] + sp[tr[k].i].rgb[ch] * tr[k].alpha * tr[k].T;
  for (size_t k = 0; k < tr.size(); ++k) {
    const Contrib& e = tr[k];
    const Splat<double>& g = sp[e.i];
    double ga = 0.0;
    for (int ch = 0; ch < 3; ++ch)
      ga += w[ch] * (g.rgb[ch] * e.T - suffix[3 * (k + 1) + ch] / (1.0 - e.alpha));
    double* c = cot + (long)e.i * NQ;
    c[Q_R] += w[0] * e.alpha * e.T;
    c[Q_G] += w[1] * e.alpha * e.T;
    c[Q_BL] += w[2] * e.alpha * e.T;
    if (e.capped) continue;
    double gpow = ga * e.alpha;
    c[Q_O] += ga * e.G;
    c[Q_A] += -0.5 * e.dx * e.dx * gpow;
    c[Q_B] += -e.dx * e.dy * gpow;
    c[Q_C] += -0.5 * e.dy * e.dy * gpow;
    c[Q_MX] += -(g.A * e.dx + g.B * e.dy) * gpow;
    c[Q_MY] += -(g.C * e.dy + g.B * e.dx) * gpow;
  }
}

// The magnitudes of the terms blend_reverse adds, with |w| in place of w: for
// every splat of the trace and every q, the absolute value of its per-pixel
// term, where dC/da's two parts (c T and the suffix over 1 - a) count by their
// absolute values.  Summed over pixels this is the mass that an FP32 sum of the
// same terms rounds against (the terms' own rounding scales with it too).
struct TraceRounding;
double tr_rel(const TraceRounding* r, size_t k);
double tr_dS(const TraceRounding* r, size_t k);
void blend_reverse_abs(const std::vector<Contrib>& tr, const std::vector<Splat<double>>& sp, const double w[3],
                       double* cot, const TraceRounding* rnd = nullptr) {
  std::vector<double> suffix(3 * (tr.size() + 1), 0.0);
  for (long k = (long)tr.size() - 1; k >= 0; --k)
    for (int ch = 0; ch < 3; ++ch)
      suffix[3 * k + ch] = suffix[3 * (k + 1) + ch] + std::fabs(sp[tr[k].i].rgb[ch]) * tr[k].alpha * tr[k].T;
  for (size_t k = 0; k < tr.size(); ++k) {
    const Contrib& e = tr[k];
    const Splat<double>& g = sp[e.i];
    double ga = 0.0, wsum = 0.0;
    for (int ch = 0; ch < 3; ++ch) {
      ga += std::fabs(w[ch]) * (std::fabs(g.rgb[ch]) * e.T + suffix[3 * (k + 1) + ch] / (1.0 - e.alpha));
      wsum += std::fabs(w[ch]);
    }
    double* c = cot + (long)e.i * NQ;
    const double f = rnd ? tr_rel(rnd, k) : 1.0;
    // with a rounding model, the suffix changes of flips behind it come on top
    if (rnd) ga += wsum * tr_dS(rnd, k) / (1.0 - e.alpha) / f;
    c[Q_R] += f * std::fabs(w[0]) * e.alpha * e.T;
    c[Q_G] += f * std::fabs(w[1]) * e.alpha * e.T;
    c[Q_BL] += f * std::fabs(w[2]) * e.alpha * e.T;
    if (e.capped) continue;
    double gpow = f * ga * e.alpha;
    c[Q_O] += f * ga * e.G;
    c[Q_A] += 0.5 * e.dx * e.dx * gpow;
    c[Q_B] += std::fabs(e.dx * e.dy) * gpow;
    c[Q_C] += 0.5 * e.dy * e.dy * gpow;
    c[Q_MX] += (std::fabs(g.A * e.dx) + std::fabs(g.B * e.dy)) * gpow;
    c[Q_MY] += (std::fabs(g.C * e.dy) + std::fabs(g.B * e.dx)) * gpow;
  }
}

// What the FP32 evaluation of each trace entry's terms may differ by, under the
// model of power_uncertainty: rel[k], relative, from its alpha's rounding (0
// when capped), the accumulated rounding of the transmittance in front of it,
// the relative change a_j / (1 - a_j) of that transmittance for every splat j in
// front of it whose own decision may flip (flips, in walk order, from
// blend_flips), and for the suffix of the splats behind it that dC/dalpha uses,
// the largest of theirs; dS[k], absolute, the change a_j T_j (c_j + c_max) of
// that suffix from the splats behind it whose decisions may flip.
struct TraceRounding {
  std::vector<double> rel, dS;
};
TraceRounding trace_rounding(const std::vector<Contrib>& tr, const std::vector<Splat<double>>& sp,
                             const std::vector<OwnFlip>& flips, double cmax) {
  TraceRounding r;
  r.rel.assign(tr.size(), 0.0);
  r.dS.assign(tr.size(), 0.0);
  auto key_less = [&](int a, int b) {
    const float da = (float)sp[a].depth, db = (float)sp[b].depth;
    return da < db || (da == db && a < b);
  };
  double tun = 0.0, front = 0.0;
  size_t f = 0;
  for (size_t k = 0; k < tr.size(); ++k) {
    const Contrib& e = tr[k];
    for (; f < flips.size() && key_less(flips[f].i, e.i); ++f) front += flips[f].a / (1.0 - flips[f].a);
    const double da = e.capped ? 0.0 : power_uncertainty(sp[e.i], e.dx, e.dy) + 2e-6;
    r.rel[k] = da + tun + front + 2e-7;
    tun += da * e.alpha / (1.0 - e.alpha) + 2e-7;
  }
  for (long k = (long)tr.size() - 2; k >= 0; --k) r.rel[k] = std::max(r.rel[k], r.rel[k + 1]);
  // suffix changes: flips behind entry k, walked back to front
  double behind = 0.0;
  long g = (long)flips.size() - 1;
  for (long k = (long)tr.size() - 1; k >= 0; --k) {
    for (; g >= 0 && key_less(tr[k].i, flips[g].i); --g) {
      const OwnFlip& q = flips[g];
      const double cq = std::max({sp[q.i].rgb[0], sp[q.i].rgb[1], sp[q.i].rgb[2], 0.0});
      behind += q.a * q.T * (cq + cmax);
    }
    r.dS[k] = behind;
  }
  return r;
}
double tr_rel(const TraceRounding* r, size_t k) { return r->rel[k]; }
double tr_dS(const TraceRounding* r, size_t k) { return r->dS[k]; }

// Parameter cotangent of splat i: sum_q cot_q d(splat_q)/d(param_r), with the
// projection Jacobian taken column by column in forward mode.
void project_reverse(const double* P, long pitch, long i, int deg, const Cam& cam, const double* cot,
                     std::vector<double>& gout /* rows values, added */) {
  int rows = n_rows(deg);
  std::vector<double> tan(rows, 0.0);
  for (int r = 0; r < rows; ++r) {
    std::fill(tan.begin(), tan.end(), 0.0);
    tan[r] = 1.0;
    G3<Dual> g = load_gaussian<Dual>(P, pitch, i, deg, tan.data());
    Splat<Dual> s = project(g, cam);
    if (!s.valid) continue;
    const double col[NQ] = {s.mx.d, s.my.d, s.A.d, s.B.d, s.C.d, s.o.d, s.rgb[0].d, s.rgb[1].d, s.rgb[2].d};
    double acc = 0.0;
    for (int q = 0; q < NQ; ++q) acc += cot[q] * col[q];
    gout[r] += acc;
  }
}

// sum_q |cot_q| |d(splat_q)/d(param_r)|: the mass of project_reverse's sums.
void project_reverse_abs(const double* P, long pitch, long i, int deg, const Cam& cam, const double* cot,
                         std::vector<double>& gout /* rows values, added */) {
  int rows = n_rows(deg);
  std::vector<double> tan(rows, 0.0);
  for (int r = 0; r < rows; ++r) {
    std::fill(tan.begin(), tan.end(), 0.0);
    tan[r] = 1.0;
    G3<Dual> g = load_gaussian<Dual>(P, pitch, i, deg, tan.data());
    Splat<Dual> s = project(g, cam);
    if (!s.valid) continue;
    const double col[NQ] = {s.mx.d, s.my.d, s.A.d, s.B.d, s.C.d, s.o.d, s.rgb[0].d, s.rgb[1].d, s.rgb[2].d};
    double acc = 0.0;
    for (int q = 0; q < NQ; ++q) acc += std::fabs(cot[q]) * std::fabs(col[q]);
    gout[r] += acc;
  }
}

// Splats of one view in forward mode along the parameter direction `dir`
// (rows x pitch).
std::vector<Splat<Dual>> project_tangent(const View& V, const double* P, long pitch, long n, int deg,
                                         const double* dir) {
  int rows = n_rows(deg);
  std::vector<Splat<Dual>> sd(n);
  std::vector<double> tan(rows);
  for (long i = 0; i < n; ++i) {
    for (int r = 0; r < rows; ++r) tan[r] = dir[(long)r * pitch + i];
    G3<Dual> g = load_gaussian<Dual>(P, pitch, i, deg, tan.data());
    sd[i] = project(g, V.cam);
  }
  return sd;
}

// Image tangent (3 x H x W) of one view for the given tangent splats.
void render_tangent(const View& V, const std::vector<Splat<Dual>>& sd, double* out) {
  long HW = (long)V.cam.W * V.cam.H;
  for_each_pixel(V, [&](int tx, int ty, int x, int y) {
    Dual C[3], T;
    int nc;
    blend(V.lists[(size_t)ty * V.Tx + tx], sd, x + 0.5, y + 0.5, C, T, nc, nullptr, nullptr);
    for (int ch = 0; ch < 3; ++ch) out[ch * HW + (long)y * V.cam.W + x] = C[ch].d;
  });
}

// ----------------------------------------------------------- trust region
// The squared Hellinger distance of Sec. 4.2, read as
//   H^2 = 1/2 (Z + Z') - sqrt(Z Z') det(S)^1/4 det(S')^1/4 / det(Sbar)^1/2
//         * exp(-1/8 dmu^T Sbar^{-1} dmu),   Sbar = (S + S') / 2,
// which equals 1/2 * integral (sqrt(G) - sqrt(G'))^2 for G = Z N(mu, S).
double det3(const double M[3][3]) {
  return M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
         M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
         M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
}
void inv3(const double M[3][3], double I[3][3]) {
  double d = det3(M);
  I[0][0] = (M[1][1] * M[2][2] - M[1][2] * M[2][1]) / d;
  I[0][1] = (M[0][2] * M[2][1] - M[0][1] * M[2][2]) / d;
  I[0][2] = (M[0][1] * M[1][2] - M[0][2] * M[1][1]) / d;
  I[1][0] = (M[1][2] * M[2][0] - M[1][0] * M[2][2]) / d;
  I[1][1] = (M[0][0] * M[2][2] - M[0][2] * M[2][0]) / d;
  I[1][2] = (M[0][2] * M[1][0] - M[0][0] * M[1][2]) / d;
  I[2][0] = (M[1][0] * M[2][1] - M[1][1] * M[2][0]) / d;
  I[2][1] = (M[0][1] * M[2][0] - M[0][0] * M[2][1]) / d;
  I[2][2] = (M[0][0] * M[1][1] - M[0][1] * M[1][0]) / d;
}

double hellinger(const double* mu1, const double* S1, double Z1, const double* mu2, const double* S2,
                 double Z2) {
  double A[3][3], B[3][3], M[3][3], Mi[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      A[a][b] = S1[3 * a + b];
      B[a][b] = S2[3 * a + b];
      M[a][b] = 0.5 * (A[a][b] + B[a][b]);
    }
  inv3(M, Mi);
  double d[3] = {mu1[0] - mu2[0], mu1[1] - mu2[1], mu1[2] - mu2[2]};
  double q = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) q += d[a] * Mi[a][b] * d[b];
  double bc = std::pow(det3(A), 0.25) * std::pow(det3(B), 0.25) / std::sqrt(det3(M)) * std::exp(-q / 8.0);
  return 0.5 * (Z1 + Z2) - std::sqrt(Z1 * Z2) * bc;
}

// Unnormalised rotation matrix R~(q) of Appendix B (entries quadratic in q).
void rot_unnorm(const double q[4], double R[3][3]) {
  double x = q[0], y = q[1], z = q[2], w = q[3];
  double r2 = x * x + y * y + z * z + w * w;
  R[0][0] = r2 - 2 * (y * y + z * z); R[0][1] = 2 * x * y - 2 * w * z; R[0][2] = 2 * x * z + 2 * w * y;
  R[1][0] = 2 * x * y + 2 * w * z; R[1][1] = r2 - 2 * (z * z + x * x); R[1][2] = 2 * y * z - 2 * w * x;
  R[2][0] = 2 * x * z - 2 * w * y; R[2][1] = 2 * y * z + 2 * w * x; R[2][2] = r2 - 2 * (x * x + y * y);
}

// beta_c of the rotation bound (Appendix B): the second derivative at a = 0 of
// T(a) = tr(S^-2 dR S^2 dR^T), dR = R(q)^T R(q + a e_c), for Sigma = R S^2 R^T:
//   beta_c = 2 || S^-1 E' S ||_F^2 + 2 tr(E''),  E' = R^T dR/dq_c,  E'' = R^T d2R/dq_c^2,
// with R = R~ / r^2, so
//   dR  = R~'/r^2 - 2 q_c R~/r^4,
//   d2R = R~''/r^2 - 4 q_c R~'/r^4 - 2 R~/r^4 + 8 q_c^2 R~/r^6.
// R~ is quadratic in q, so its first and second partial derivatives are given
// exactly by the symmetric differences (R~(q+e) - R~(q-e))/2 and R~(q+e) - 2R~(q) + R~(q-e).
void rotation_beta(const double q[4], const double s[3], double beta[4]) {
  double r2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
  double Rt[3][3], R[3][3];
  rot_unnorm(q, Rt);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) R[a][b] = Rt[a][b] / r2;
  for (int c = 0; c < 4; ++c) {
    double qp[4], qm[4];
    for (int a = 0; a < 4; ++a) { qp[a] = q[a]; qm[a] = q[a]; }
    qp[c] += 1.0; qm[c] -= 1.0;
    double Rp[3][3], Rm[3][3], d1[3][3], d2[3][3], dR[3][3], ddR[3][3];
    rot_unnorm(qp, Rp);
    rot_unnorm(qm, Rm);
    double qc = q[c];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        d1[a][b] = 0.5 * (Rp[a][b] - Rm[a][b]);
        d2[a][b] = Rp[a][b] - 2.0 * Rt[a][b] + Rm[a][b];
        dR[a][b] = d1[a][b] / r2 - 2.0 * qc * Rt[a][b] / (r2 * r2);
        ddR[a][b] = d2[a][b] / r2 - 4.0 * qc * d1[a][b] / (r2 * r2) - 2.0 * Rt[a][b] / (r2 * r2) +
                    8.0 * qc * qc * Rt[a][b] / (r2 * r2 * r2);
      }
    double E1[3][3], E2[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        E1[a][b] = E2[a][b] = 0.0;
        for (int u = 0; u < 3; ++u) {
          E1[a][b] += R[u][a] * dR[u][b];
          E2[a][b] += R[u][a] * ddR[u][b];
        }
      }
    double fro = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double m = E1[a][b] * s[b] / s[a];  // (S^-1 E' S)_ab
        fro += m * m;
      }
    beta[c] = 2.0 * fro + 2.0 * (E2[0][0] + E2[1][1] + E2[2][2]);
  }
}

// max over the unit sphere of |Y_k|, by a dense grid search refined by a local
// pattern search.
void sh_absmax(int deg, double* ymax) {
  int K = n_coeffs(deg);
  auto f = [&](int k, double th, double ph) {
    double Y[16];
    sh_basis<double>(deg, std::sin(th) * std::cos(ph), std::sin(th) * std::sin(ph), std::cos(th), Y);
    return std::fabs(Y[k]);
  };
  const int NT = 400, NP = 800;
  for (int k = 0; k < K; ++k) {
    double best = -1.0, bt = 0.0, bp = 0.0;
    for (int a = 0; a <= NT; ++a)
      for (int b = 0; b < NP; ++b) {
        double th = kPi * a / NT, ph = 2.0 * kPi * b / NP;
        double v = f(k, th, ph);
        if (v > best) { best = v; bt = th; bp = ph; }
      }
    double step = kPi / NT;
    while (step > 1e-10) {
      bool moved = false;
      for (int dt = -1; dt <= 1; ++dt)
        for (int dp = -1; dp <= 1; ++dp) {
          double v = f(k, bt + dt * step, bp + dp * step);
          if (v > best) { best = v; bt += dt * step; bp += dp * step; moved = true; }
        }
      if (!moved) step *= 0.5;
    }
    ymax[k] = best;
  }
}

struct TRConfig {
  double theta1, theta2, d_floor, color_floor;
  int l, mean_exact;
};

TRConfig read_cfg(const double* c) {
  TRConfig k;
  k.theta1 = c[0]; k.theta2 = c[1]; k.d_floor = c[2]; k.color_floor = c[3];
  k.l = (int)c[4]; k.mean_exact = (int)c[5];
  return k;
}

const double kInf = std::numeric_limits<double>::infinity();

// Per-parameter radius eta = SHD(x, eps) of every parameter of splat i (Sec. 4.2,
// Appendix B), mapped to this parameterisation by the first-order chain rule:
//   mean        sqrt(-8 Sigma_cc ln(1 - eps/alpha))      (inf when alpha <= eps)
//   log-scale   sqrt(2 eps / alpha)                       (|dS_c| < sqrt(2 S_c^2 eps/alpha), dS = S dlogS)
//   quaternion  sqrt(-(8/beta_c) ln(1 - eps/alpha))       (inf when beta_c = 0 or alpha <= eps)
//   logit       sqrt(4 alpha eps) / (alpha (1 - alpha))   (d alpha = alpha (1 - alpha) d logit)
//   SH (k, c)   sqrt(4 C_c eps / alpha) / max|Y_k|        (C_c = DC colour, floored)
void shd_radius(const double* P, long pitch, long i, int deg, double eps, const TRConfig& cfg,
                const double* ymax, double* eta) {
  int K = n_coeffs(deg);
  G3<double> g = load_gaussian<double>(P, pitch, i, deg, nullptr);
  double alpha = 1.0 / (1.0 + std::exp(-g.ol));
  double s[3], R[3][3], Sig[3][3];
  for (int a = 0; a < 3; ++a) s[a] = std::exp(g.ls[a]);
  rotmat<double>(g.q, R);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      Sig[a][b] = R[a][0] * s[0] * s[0] * R[b][0] + R[a][1] * s[1] * s[1] * R[b][1] +
                  R[a][2] * s[2] * s[2] * R[b][2];
  double Si[3][3];
  inv3(Sig, Si);
  bool logok = alpha > eps;
  double L = logok ? std::log1p(-eps / alpha) : 0.0;
  for (int c = 0; c < 3; ++c) {
    double var = cfg.mean_exact ? 1.0 / Si[c][c] : Sig[c][c];
    eta[c] = logok ? std::sqrt(-8.0 * var * L) : kInf;
    eta[3 + c] = std::sqrt(2.0 * eps / alpha);
  }
  double beta[4];
  rotation_beta(g.q, s, beta);
  for (int c = 0; c < 4; ++c) eta[6 + c] = (logok && beta[c] > 0.0) ? std::sqrt(-8.0 / beta[c] * L) : kInf;
  eta[10] = std::sqrt(4.0 * alpha * eps) / (alpha * (1.0 - alpha));
  const double c0 = 0.5 * std::sqrt(1.0 / kPi);
  for (int ch = 0; ch < 3; ++ch) {
    double Cc = std::max(c0 * g.sh[0][ch] + 0.5, cfg.color_floor);
    for (int k = 0; k < K; ++k) eta[kRowSH + 3 * k + ch] = std::sqrt(4.0 * Cc * eps / alpha) / ymax[k];
  }
}

struct Scene {
  const double* P;
  long pitch, n;
  int deg;
};

}  // namespace

// ======================================================================= C ABI
extern "C" {

uint64_t or_splitmix64(uint64_t x) { return splitmix64(x); }

double or_rademacher(uint64_t seed, int64_t t, int k, uint64_t j) { return rademacher(seed, t, k, j); }

void or_sh_basis(int deg, const double* dir, double* Y) {
  double n = std::sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
  sh_basis<double>(deg, dir[0] / n, dir[1] / n, dir[2] / n, Y);
}

void or_sh_absmax(int deg, double* ymax) { sh_absmax(deg, ymax); }

void or_quat_to_rotmat(const double* q, double* R9) {
  double R[3][3];
  rotmat<double>(q, R);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) R9[3 * a + b] = R[a][b];
}

// Projection of every splat for one camera.  out: n x 13 doubles
//   mx, my, A, B, C, o, r, g, b, depth, radius_raw, radius, valid
void or_project(const double* P, long pitch, long n, int deg, const double* cam24, double* out) {
  Cam cam = make_cam(cam24);
  for (long i = 0; i < n; ++i) {
    Splat<double> s = project(load_gaussian<double>(P, pitch, i, deg, nullptr), cam);
    double* o = out + 13 * i;
    double v[13] = {s.mx, s.my, s.A, s.B, s.C, s.o, s.rgb[0], s.rgb[1], s.rgb[2], s.depth,
                    s.radius_raw, (double)(s.valid ? s.radius : 0), s.valid ? 1.0 : 0.0};
    if (!s.valid) for (int q = 0; q < 10; ++q) v[q] = 0.0;
    std::memcpy(o, v, sizeof(v));
  }
}

// Selects the tiles of a splat in every later render, JVP, Jacobian and backward
// call: 0 (the default) its 3DGS square, 1 the square narrowed to its footprint box.
void or_set_footprint_bins(int on) { g_footprint_bins = on ? 1 : 0; }

// Binning and depth sort from FP32 splat records of n_views views (arrays are
// n_views x n; A, B, C the conic).  `ext` holds each record's footprint
// half-extents as packed halves (x low, y high); null bins by the 3DGS square.  Writes up to `cap` pairs and the [start, end) range of every
// tile (2 x n_views x tiles); returns the number of pairs.
long or_bin_sort(int n_views, long n, const float* mx, const float* my, const float* A, const float* B,
                 const float* C, const int* rad, const uint32_t* ext, const float* depth, int W, int H, int tw,
                 int th, uint64_t* keys, uint32_t* vals, long cap, uint32_t* ranges) {
  std::vector<float> hx((size_t)n_views * n, INFINITY), hy((size_t)n_views * n, INFINITY);
  if (ext)
    for (long g = 0; g < (long)n_views * n; ++g) {
      hx[g] = half_to_float((uint16_t)(ext[g] & 0xffffu));
      hy[g] = half_to_float((uint16_t)(ext[g] >> 16));
    }
  std::vector<Pair> pairs =
      bin_and_sort(n_views, n, mx, my, A, B, C, rad, hx.data(), hy.data(), depth, W, H, tw, th, ext != nullptr);
  long T = (long)((W + tw - 1) / tw) * ((H + th - 1) / th);
  for (long k = 0; k < 2 * T * n_views; ++k) ranges[k] = 0;
  for (long p = 0; p < (long)pairs.size(); ++p) {
    if (p < cap) { keys[p] = pairs[p].key; vals[p] = pairs[p].val; }
    uint64_t tile = pairs[p].key >> 32;
    if (p == 0 || (pairs[p - 1].key >> 32) != tile) ranges[2 * tile] = (uint32_t)p;
    ranges[2 * tile + 1] = (uint32_t)(p + 1);
  }
  return (long)pairs.size();
}

// Render every view.  image: V x 3 x H x W, final_T and margin: V x H x W,
// n_contrib: V x H x W.  margin is the smallest relative distance of a threshold
// decision at the pixel, or 0 where binning is within rounding of a boundary.
// impact, t_impact, err (V x H x W, may be null): the bounds of blend_flips on
// what FP32 decision flips can do to the colour and the final T, and on the
// colour's own rounding; nc_range (V x H x W x 2, may be null): the n_contrib
// values those flips and the tile sets within rounding allow.  Returns the
// total number of (tile, splat) pairs.
long or_render(const double* P, long pitch, long n, int deg, const double* cams, int n_views, int tw, int th,
               double* image, double* final_T, int32_t* n_contrib, double* margin, int32_t* nc_range,
               double* impact, double* t_impact, double* err) {
  long pairs = 0;
  for (int v = 0; v < n_views; ++v) {
    View V = build_view(P, pitch, n, deg, cams + 24 * v, tw, th);
    long HW = (long)V.cam.W * V.cam.H;
    for (const auto& l : V.lists) pairs += (long)l.size();
    double* img = image + v * 3 * HW;
    for_each_pixel(V, [&](int tx, int ty, int x, int y) {
      double C[3], T, mg;
      int nc;
      blend(V.lists[(size_t)ty * V.Tx + tx], V.sp, x + 0.5, y + 0.5, C, T, nc, &mg, nullptr);
      long px = (long)y * V.cam.W + x;
      for (int ch = 0; ch < 3; ++ch) img[ch * HW + px] = C[ch];
      final_T[v * HW + px] = T;
      n_contrib[v * HW + px] = nc;
      int lo = nc, hi = nc;
      if (margin)
        margin[v * HW + px] = std::min(mg, binning_margin(V, tx, ty, x + 0.5, y + 0.5, nc, &lo, &hi));
      if (impact || nc_range || err) {
        const size_t tile = (size_t)ty * V.Tx + tx;
        const Flip fl = blend_flips(V, tile, x + 0.5, y + 0.5, nc);
        if (impact) impact[v * HW + px] = fl.impact;
        if (t_impact) t_impact[v * HW + px] = fl.t_impact;
        if (err) err[v * HW + px] = fl.err;
        lo = fl.nc_lo;
        hi = fl.nc_hi;
      }
      if (nc_range) {
        nc_range[2 * (v * HW + px)] = lo;
        nc_range[2 * (v * HW + px) + 1] = hi;
      }
    });
  }
  return pairs;
}

// Forward-mode tangents of the splat quantities (mx, my, A, B, C, o, r, g, b) of
// every Gaussian for one camera along the parameter direction `dir`
// (rows x pitch).  out: n x 9.
void or_project_tangent(const double* P, long pitch, long n, int deg, const double* cam24, const double* dir,
                        double* out) {
  Cam cam = make_cam(cam24);
  int rows = n_rows(deg);
  std::vector<double> tan(rows);
  for (long i = 0; i < n; ++i) {
    for (int r = 0; r < rows; ++r) tan[r] = dir[(long)r * pitch + i];
    Splat<Dual> s = project(load_gaussian<Dual>(P, pitch, i, deg, tan.data()), cam);
    double v[9] = {s.mx.d, s.my.d, s.A.d, s.B.d, s.C.d, s.o.d, s.rgb[0].d, s.rgb[1].d, s.rgb[2].d};
    if (!s.valid) for (int q = 0; q < 9; ++q) v[q] = 0.0;
    std::memcpy(out + 9 * i, v, sizeof(v));
  }
}

// Image tangent (V x 3 x H x W) along the parameter direction `dir` (rows x pitch).
void or_jvp(const double* P, long pitch, long n, int deg, const double* cams, int n_views, int tw, int th,
            const double* dir, double* img_tan) {
  long off = 0;
  for (int v = 0; v < n_views; ++v) {
    View V = build_view(P, pitch, n, deg, cams + 24 * v, tw, th);
    std::vector<Splat<Dual>> sd = project_tangent(V, P, pitch, n, deg, dir);
    render_tangent(V, sd, img_tan + off);
    off += 3L * V.cam.W * V.cam.H;
  }
}

// Full image Jacobian dC/dx for tiny scenes: J has (sum_v 3 H W) rows and
// (rows * n) columns, column index r * n + i, row-major.
void or_jacobian(const double* P, long pitch, long n, int deg, const double* cams, int n_views, int tw,
                 int th, double* J) {
  int rows = n_rows(deg);
  long ncol = (long)rows * n;
  std::vector<double> dir((size_t)rows * pitch, 0.0);
  long total = 0;
  for (int v = 0; v < n_views; ++v) {
    Cam c = make_cam(cams + 24 * v);
    total += 3L * c.W * c.H;
  }
  std::vector<double> col(total);
  for (int r = 0; r < rows; ++r)
    for (long i = 0; i < n; ++i) {
      dir[(size_t)r * pitch + i] = 1.0;
      or_jvp(P, pitch, n, deg, cams, n_views, tw, th, dir.data(), col.data());
      dir[(size_t)r * pitch + i] = 0.0;
      long cidx = (long)r * n + i;
      for (long k = 0; k < total; ++k) J[k * ncol + cidx] = col[k];
    }
}

// One backward + Hutchinson pass over `n_views` views with targets (V x 3 x H x W).
//   loss_kind 0: F = sqrt(|r|) (L1), dL/dC = sign(r)/(2m), GN weight 1/(4 max(|r|, gn_floor));
//   loss_kind 1: F = r (L2),          dL/dC = r/m,          GN weight 1.
// m = sum over views of 3 H W.  grad (rows x n, row pitch n) receives g = (1/m) J^T F.
// If nu > 0, hz (rows x n) receives (1/nu) sum_k z_k . ((1/m) J^T diag(w) J z_k) with the
// Rademacher probes of (seed, t, k), and img_tan (nu x V x 3 x H x W, may be null) the
// tangents J z_k.  res_margin (V x H x W, may be null) receives min over channels of |r|.
// Returns the objective f = (1/2m) sum F^2.
//   loss_kind 2 (or_backward_dssim): per pixel and channel the two components
//     F = sqrt((1 - lambda) |r|) and F = sqrt(lambda (1 - S)) (Eq. pixel_loss
//     with D-SSIM = 1 - S), m = sum over views of 6 H W; dL/dC = (1/2m)
//     ((1 - lambda) sign(r) - lambda sum_p dS_p/dC), and the Gauss-Newton
//     vector of probe k is (1 - lambda)/(4 max(|r|, gn_floor))/m . J z_k plus
//     the adjoint of S applied to lambda/(4 max(1 - S, gn_floor))/m . dS[J z_k].
// grad_mass, hz_mass (rows x n, may be null): per entry, the mass of the sum
// that forms it (blend_reverse_abs over every pixel, then project_reverse_abs),
// the scale an FP32 evaluation of the same sums rounds against.  hz_sens (rows
// x n, may be null; L1 only): the bound of or_backward_sampled on how far the
// Hutchinson entries move when each residual moves by its pixel's FP32 rounding
// bound or by the image tolerance kImageTol, whichever is smaller.
double backward_impl(const double* P, long pitch, long n, int deg, const double* cams, int n_views, int tw,
                     int th, const double* target, int loss_kind, double lambda, double gn_floor, uint64_t seed,
                     int64_t t, int nu, double* grad, double* hz, double* img_tan, double* res_margin,
                     double* grad_mass, double* hz_mass, double* hz_sens = nullptr, double* grad_allow = nullptr,
                     double* hz_allow = nullptr, double* grad_round = nullptr, double* hz_round = nullptr) {
  int rows = n_rows(deg);
  double m = 0.0;
  std::vector<View> views;
  for (int v = 0; v < n_views; ++v) {
    views.push_back(build_view(P, pitch, n, deg, cams + 24 * v, tw, th));
    m += (loss_kind == 2 ? 6.0 : 3.0) * views.back().cam.W * views.back().cam.H;
  }
  for (long k = 0; k < (long)rows * n; ++k) grad[k] = 0.0;
  if (hz) for (long k = 0; k < (long)rows * n; ++k) hz[k] = 0.0;
  const bool masses = grad_mass != nullptr;
  if (grad_mass) for (long k = 0; k < (long)rows * n; ++k) grad_mass[k] = 0.0;
  if (hz_mass) for (long k = 0; k < (long)rows * n; ++k) hz_mass[k] = 0.0;
  if (hz_sens) for (long k = 0; k < (long)rows * n; ++k) hz_sens[k] = 0.0;
  if (grad_allow) for (long k = 0; k < (long)rows * n; ++k) grad_allow[k] = 0.0;
  if (hz_allow) for (long k = 0; k < (long)rows * n; ++k) hz_allow[k] = 0.0;
  if (grad_round) for (long k = 0; k < (long)rows * n; ++k) grad_round[k] = 0.0;
  if (hz_round) for (long k = 0; k < (long)rows * n; ++k) hz_round[k] = 0.0;
  const bool sensing = hz_sens != nullptr && loss_kind == 0 && nu > 0;
  const bool allowing = grad_allow != nullptr;

  // probe directions z_k over the parameter vector (entry i * rows + r)
  std::vector<std::vector<double>> z(nu, std::vector<double>((size_t)rows * pitch, 0.0));
  for (int k = 0; k < nu; ++k)
    for (int r = 0; r < rows; ++r)
      for (long i = 0; i < n; ++i) z[k][(size_t)r * pitch + i] = rademacher(seed, t, k, probe_entry(i, r, rows));

  long total = 0;  // sum over views of 3 H W
  for (const View& V : views) total += 3L * V.cam.W * V.cam.H;
  double f = 0.0;
  long img_off = 0;
  std::vector<double> g_acc(rows);
  for (int v = 0; v < n_views; ++v) {
    const View& V = views[v];
    long HW = (long)V.cam.W * V.cam.H;
    const double* tg = target + img_off;
    // streams: 0 = gradient, 1..nu = Gauss-Newton products
    std::vector<std::vector<double>> cot(1 + nu, std::vector<double>((size_t)n * NQ, 0.0));
    std::vector<std::vector<double>> cot_abs(masses ? 1 + nu : 0, std::vector<double>((size_t)n * NQ, 0.0));
    std::vector<std::vector<double>> cot_sens(sensing ? nu : 0, std::vector<double>((size_t)n * NQ, 0.0));
    std::vector<std::vector<double>> cot_allow(allowing ? 1 + nu : 0, std::vector<double>((size_t)n * NQ, 0.0));
    std::vector<std::vector<double>> cot_round(allowing ? 1 + nu : 0, std::vector<double>((size_t)n * NQ, 0.0));
    std::vector<OwnFlip> ofl;
    TraceRounding trel;
    std::vector<std::vector<double>> jz(nu, std::vector<double>(3 * HW, 0.0));
    for (int k = 0; k < nu; ++k) {
      std::vector<Splat<Dual>> sd = project_tangent(V, P, pitch, n, deg, z[k].data());
      render_tangent(V, sd, jz[k].data());
      if (img_tan) std::memcpy(img_tan + (long)k * total + img_off, jz[k].data(), 3 * HW * sizeof(double));
    }
    // D-SSIM: the whole image's cotangents first (SSIM couples neighbouring pixels)
    std::vector<double> cw, cu;
    if (loss_kind == 2) {
      const int H = V.cam.H, W = V.cam.W;
      std::vector<double> img(3 * HW, 0.0);
      for_each_pixel(V, [&](int tx, int ty, int x, int y) {
        double C[3], T;
        int nc;
        blend(V.lists[(size_t)ty * V.Tx + tx], V.sp, x + 0.5, y + 0.5, C, T, nc, nullptr, nullptr);
        for (int ch = 0; ch < 3; ++ch) img[ch * HW + (long)y * W + x] = C[ch];
      });
      cw.assign(3 * HW, 0.0);
      cu.assign((size_t)nu * 3 * HW, 0.0);
      std::vector<double> ones(HW, 1.0), a(HW);
      for (int ch = 0; ch < 3; ++ch) {
        const double* xc = img.data() + ch * HW;
        const double* yc = tg + ch * HW;
        SsimMaps M = ssim_maps(xc, yc, H, W);
        std::vector<double> gS = ssim_vjp(xc, yc, H, W, M, ones.data());
        for (long px = 0; px < HW; ++px) {
          const double r = xc[px] - yc[px];
          f += ((1.0 - lambda) * std::fabs(r) + lambda * (1.0 - M.S[px])) / (2.0 * m);
          cw[ch * HW + px] = ((1.0 - lambda) * (r > 0 ? 1.0 : (r < 0 ? -1.0 : 0.0)) - lambda * gS[px]) / (2.0 * m);
        }
        for (int k = 0; k < nu; ++k) {
          const double* d = jz[k].data() + ch * HW;
          std::vector<double> dS = ssim_jvp(xc, yc, H, W, M, d);
          for (long px = 0; px < HW; ++px) a[px] = lambda / (4.0 * std::max(1.0 - M.S[px], gn_floor)) / m * dS[px];
          std::vector<double> back = ssim_vjp(xc, yc, H, W, M, a.data());
          for (long px = 0; px < HW; ++px) {
            const double r = xc[px] - yc[px];
            cu[((size_t)k * 3 + ch) * HW + px] =
                (1.0 - lambda) / (4.0 * std::max(std::fabs(r), gn_floor)) / m * d[px] + back[px];
          }
        }
      }
    }
    for_each_pixel(V, [&](int tx, int ty, int x, int y) {
      double C[3], T;
      int nc;
      std::vector<Contrib> tr;
      blend(V.lists[(size_t)ty * V.Tx + tx], V.sp, x + 0.5, y + 0.5, C, T, nc, nullptr, &tr);
      long px = (long)y * V.cam.W + x;
      double w[3], wgn[3], rmin = kInf;
      for (int ch = 0; ch < 3; ++ch) {
        double r = C[ch] - tg[ch * HW + px];
        rmin = std::min(rmin, std::fabs(r));
        if (loss_kind == 2) {
          w[ch] = cw[ch * HW + px];
          wgn[ch] = 0.0;  // the probe vectors come whole from cu
        } else if (loss_kind == 0) {
          f += std::fabs(r) / (2.0 * m);
          w[ch] = (r > 0 ? 1.0 : (r < 0 ? -1.0 : 0.0)) / (2.0 * m);
          wgn[ch] = 1.0 / (4.0 * std::max(std::fabs(r), gn_floor)) / m;
        } else {
          f += r * r / (2.0 * m);
          w[ch] = r / m;
          wgn[ch] = 1.0 / m;
        }
      }
      if (res_margin) res_margin[v * HW + px] = rmin;
      blend_reverse(tr, V.sp, w, cot[0].data());
      if (masses) blend_reverse_abs(tr, V.sp, w, cot_abs[0].data());
      double sens[3] = {0.0, 0.0, 0.0};
      const size_t tile = (size_t)ty * V.Tx + tx;
      ofl.clear();
      // how far the GPU's residual here may be from the oracle's: its colour's
      // rounding (capped at the image tolerance) plus what decision flips do to it
      double e_res = 0.0;
      if (sensing || allowing) {
        const Flip fl = blend_flips(V, tile, x + 0.5, y + 0.5, nc, allowing ? &ofl : nullptr);
        e_res = std::min(fl.err, kImageTol) + fl.impact;
        for (int ch = 0; sensing && ch < 3; ++ch) {
          const double r = std::fabs(C[ch] - tg[ch * HW + px]);
          sens[ch] = r + e_res > gn_floor ? e_res / std::max(r, gn_floor) : 0.0;
        }
      }
      if (allowing) {
        // own decisions that may flip here, and dL/dC's own uncertainty: (L1) a
        // residual sign within e_res changes it by 2 |w|, (L2) w = r/m moves by e_res/m
        for (const OwnFlip& q : ofl) own_terms(V.sp[q.i], q, V.tile_cmax[tile], w, cot_allow[0].data() + q.i * NQ);
        double wflip[3];
        for (int ch = 0; ch < 3; ++ch) {
          const double r = std::fabs(C[ch] - tg[ch * HW + px]);
          wflip[ch] = loss_kind == 0 ? (r < e_res ? 2.0 * w[ch] : 0.0) : (loss_kind == 1 ? e_res / m : 0.0);
        }
        blend_reverse_abs(tr, V.sp, wflip, cot_allow[0].data());
        trel = trace_rounding(tr, V.sp, ofl, V.tile_cmax[tile]);
        blend_reverse_abs(tr, V.sp, w, cot_round[0].data(), &trel);
      }
      for (int k = 0; k < nu; ++k) {
        double wk[3];
        for (int ch = 0; ch < 3; ++ch)
          wk[ch] = loss_kind == 2 ? cu[((size_t)k * 3 + ch) * HW + px] : wgn[ch] * jz[k][ch * HW + px];
        blend_reverse(tr, V.sp, wk, cot[1 + k].data());
        if (masses) blend_reverse_abs(tr, V.sp, wk, cot_abs[1 + k].data());
        if (sensing) {
          double ws[3];
          for (int ch = 0; ch < 3; ++ch) ws[ch] = wk[ch] * sens[ch];
          blend_reverse_abs(tr, V.sp, ws, cot_sens[k].data());
        }
        if (allowing) {
          for (const OwnFlip& q : ofl)
            own_terms(V.sp[q.i], q, V.tile_cmax[tile], wk, cot_allow[1 + k].data() + q.i * NQ);
          blend_reverse_abs(tr, V.sp, wk, cot_round[1 + k].data(), &trel);
        }
      }
    });
    for (long i = 0; i < n; ++i) {
      if (!V.sp[i].valid) continue;
      for (int s = 0; s <= nu; ++s) {
        const double* c = cot[s].data() + i * NQ;
        bool any = false;
        for (int q = 0; q < NQ; ++q)
          any = any || c[q] != 0.0 || (allowing && (cot_allow[s][(size_t)i * NQ + q] != 0.0 ||
                                                    cot_round[s][(size_t)i * NQ + q] != 0.0));
        if (!any) continue;
        std::fill(g_acc.begin(), g_acc.end(), 0.0);
        project_reverse(P, pitch, i, deg, V.cam, c, g_acc);
        for (int r = 0; r < rows; ++r) {
          if (s == 0) grad[(long)r * n + i] += g_acc[r];
          else hz[(long)r * n + i] += z[s - 1][(size_t)r * pitch + i] * g_acc[r] / nu;
        }
        if (sensing && s > 0) {
          std::fill(g_acc.begin(), g_acc.end(), 0.0);
          project_reverse_abs(P, pitch, i, deg, V.cam, cot_sens[s - 1].data() + i * NQ, g_acc);
          for (int r = 0; r < rows; ++r) hz_sens[(long)r * n + i] += g_acc[r] / nu;
        }
        if (allowing && (s == 0 || hz_allow)) {
          std::fill(g_acc.begin(), g_acc.end(), 0.0);
          project_reverse_abs(P, pitch, i, deg, V.cam, cot_allow[s].data() + i * NQ, g_acc);
          for (int r = 0; r < rows; ++r) (s == 0 ? grad_allow : hz_allow)[(long)r * n + i] += g_acc[r] / (s == 0 ? 1 : nu);
        }
        double* rout = s == 0 ? grad_round : hz_round;
        if (allowing && rout) {
          std::fill(g_acc.begin(), g_acc.end(), 0.0);
          project_reverse_abs(P, pitch, i, deg, V.cam, cot_round[s].data() + i * NQ, g_acc);
          for (int r = 0; r < rows; ++r) rout[(long)r * n + i] += g_acc[r] / (s == 0 ? 1 : nu);
        }
        if (!masses || (s > 0 && !hz_mass)) continue;
        std::fill(g_acc.begin(), g_acc.end(), 0.0);
        project_reverse_abs(P, pitch, i, deg, V.cam, cot_abs[s].data() + i * NQ, g_acc);
        for (int r = 0; r < rows; ++r) {
          if (s == 0) grad_mass[(long)r * n + i] += g_acc[r];
          else hz_mass[(long)r * n + i] += g_acc[r] / nu;
        }
      }
    }
    img_off += 3 * HW;
  }
  return f;
}

double or_backward(const double* P, long pitch, long n, int deg, const double* cams, int n_views, int tw,
                   int th, const double* target, int loss_kind, double gn_floor, uint64_t seed, int64_t t,
                   int nu, double* grad, double* hz, double* img_tan, double* res_margin, double* grad_mass,
                   double* hz_mass, double* hz_sens, double* grad_allow, double* hz_allow, double* grad_round,
                   double* hz_round) {
  return backward_impl(P, pitch, n, deg, cams, n_views, tw, th, target, loss_kind, 0.0, gn_floor, seed, t, nu,
                       grad, hz, img_tan, res_margin, grad_mass, hz_mass, hz_sens, grad_allow, hz_allow, grad_round,
                       hz_round);
}

double or_backward_dssim(const double* P, long pitch, long n, int deg, const double* cams, int n_views, int tw,
                         int th, const double* target, double lambda, double gn_floor, uint64_t seed, int64_t t,
                         int nu, double* grad, double* hz, double* img_tan, double* grad_mass, double* hz_mass,
                         double* grad_allow, double* hz_allow, double* grad_round, double* hz_round) {
  return backward_impl(P, pitch, n, deg, cams, n_views, tw, th, target, 2, lambda, gn_floor, seed, t, nu, grad, hz,
                       img_tan, nullptr, grad_mass, hz_mass, nullptr, grad_allow, hz_allow, grad_round, hz_round);
}

// SSIM map of one channel and its partials (for the pins), and the adjoint and
// directional derivative of the map.
void or_ssim(const double* x, const double* y, int H, int W, double* S, double* dmx, double* dex2, double* dexy) {
  SsimMaps M = ssim_maps(x, y, H, W);
  std::copy(M.S.begin(), M.S.end(), S);
  if (dmx) std::copy(M.dmx.begin(), M.dmx.end(), dmx);
  if (dex2) std::copy(M.dex2.begin(), M.dex2.end(), dex2);
  if (dexy) std::copy(M.dexy.begin(), M.dexy.end(), dexy);
}
void or_ssim_vjp(const double* x, const double* y, int H, int W, const double* a, double* out) {
  SsimMaps M = ssim_maps(x, y, H, W);
  std::vector<double> g = ssim_vjp(x, y, H, W, M, a);
  std::copy(g.begin(), g.end(), out);
}
void or_ssim_jvp(const double* x, const double* y, int H, int W, const double* d, double* out) {
  SsimMaps M = ssim_maps(x, y, H, W);
  std::vector<double> g = ssim_jvp(x, y, H, W, M, d);
  std::copy(g.begin(), g.end(), out);
}

// Per-parameter trust-region radii (rows x n, row pitch n).
// cfg: theta1, theta2, d_floor, color_floor, l, mean_exact.
void or_shd_radius(const double* P, long pitch, long n, int deg, double eps, const double* cfg6,
                   double* eta) {
  TRConfig cfg = read_cfg(cfg6);
  int rows = n_rows(deg);
  double ymax[16];
  sh_absmax(deg, ymax);
  std::vector<double> e(rows);
  for (long i = 0; i < n; ++i) {
    shd_radius(P, pitch, i, deg, eps, cfg, ymax, e.data());
    for (int r = 0; r < rows; ++r) eta[(long)r * n + i] = e[r];
  }
}

// Algorithm 1, lines "update EMA of g", "update EMA of D every l steps", Newton
// step, radius, clip, update, for step t (t >= 1).  Arrays are rows x pitch;
// hz may be null on steps without a Hutchinson estimate.  The denominator is
// max(D_hat, d_floor).  If eta_out is given it receives the radii (rows x pitch).
void or_tr_update(double* x, double* g_ema, double* d_ema, const double* grad, const double* hz, long pitch,
                  long n, int deg, const double* cfg6, int64_t t, double eps, double* eta_out) {
  TRConfig cfg = read_cfg(cfg6);
  int rows = n_rows(deg);
  double ymax[16];
  sh_absmax(deg, ymax);
  bool hvp_step = ((t - 1) % cfg.l) == 0;
  std::vector<double> eta(rows);
  for (long i = 0; i < n; ++i) {
    shd_radius(x, pitch, i, deg, eps, cfg, ymax, eta.data());  // from x_t, before the update
    for (int r = 0; r < rows; ++r) {
      long j = (long)r * pitch + i;
      g_ema[j] = cfg.theta1 * g_ema[j] + (1.0 - cfg.theta1) * grad[j];
      if (hvp_step && hz) d_ema[j] = cfg.theta2 * d_ema[j] + (1.0 - cfg.theta2) * hz[j];
      double delta = -g_ema[j] / std::max(d_ema[j], cfg.d_floor);
      double e = eta[r];
      double dh = std::min(std::max(delta, -e), e);
      if (eta_out) eta_out[j] = e;
      x[j] += dh;
    }
  }
}

// ADAM-TR (Sec. 5, ablation): the Hellinger trust-region clip of Sec. 4.2
// applied to an Adam step instead of the Newton step.  For step t >= 1, per
// parameter j of row group q (mean, log-scale, quaternion, opacity, SH DC, SH
// rest; adam9 = beta1, beta2, eps_adam, lr[q] for q = 0..5):
//   m = beta1 m + (1 - beta1) g,   v = beta2 v + (1 - beta2) g^2
//   delta = -lr[q] (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps_adam)
//   x += clip(delta, -eta, eta), eta the radius of x_t as in or_tr_update.
void or_adam_tr_update(double* x, double* m, double* v, const double* grad, long pitch, long n, int deg,
                       const double* cfg6, const double* adam9, int64_t t, double eps, double* eta_out) {
  TRConfig cfg = read_cfg(cfg6);
  int rows = n_rows(deg);
  double ymax[16];
  sh_absmax(deg, ymax);
  const double b1 = adam9[0], b2 = adam9[1], ea = adam9[2];
  const double bc1 = 1.0 - std::pow(b1, (double)t), bc2 = 1.0 - std::pow(b2, (double)t);
  std::vector<double> eta(rows);
  for (long i = 0; i < n; ++i) {
    shd_radius(x, pitch, i, deg, eps, cfg, ymax, eta.data());  // from x_t, before the update
    for (int r = 0; r < rows; ++r) {
      const int q = r < 3 ? 0 : r < 6 ? 1 : r < 10 ? 2 : r < 11 ? 3 : r < 14 ? 4 : 5;
      long j = (long)r * pitch + i;
      m[j] = b1 * m[j] + (1.0 - b1) * grad[j];
      v[j] = b2 * v[j] + (1.0 - b2) * grad[j] * grad[j];
      double delta = -adam9[3 + q] * (m[j] / bc1) / (std::sqrt(v[j] / bc2) + ea);
      double e = eta[r];
      if (eta_out) eta_out[j] = e;
      x[j] += std::min(std::max(delta, -e), e);
    }
  }
}

// Per-pixel signature (V x H x W) of every discrete decision the blend took:
// which splats contributed, whether their alpha was capped, and which clamps of
// their projection were active.  Two parameter vectors with equal signatures
// lie on the same smooth piece of the objective.
void or_signature(const double* P, long pitch, long n, int deg, const double* cams, int n_views, int tw,
                  int th, uint64_t* sig) {
  long off = 0;
  for (int v = 0; v < n_views; ++v) {
    View V = build_view(P, pitch, n, deg, cams + 24 * v, tw, th);
    for_each_pixel(V, [&](int tx, int ty, int x, int y) {
      double C[3], T;
      int nc;
      std::vector<Contrib> tr;
      blend(V.lists[(size_t)ty * V.Tx + tx], V.sp, x + 0.5, y + 0.5, C, T, nc, nullptr, &tr);
      uint64_t h = 0xcbf29ce484222325ULL;
      auto mix = [&](uint64_t u) { h = (h ^ u) * 0x100000001b3ULL; };
      for (const Contrib& e : tr) {
        mix((uint64_t)e.i);
        mix((uint64_t)(e.capped ? 1 : 0) | ((uint64_t)V.sp[e.i].flags << 1));
      }
      mix((uint64_t)nc);
      sig[off + (long)y * V.cam.W + x] = h;
    });
    off += (long)V.cam.W * V.cam.H;
  }
}

// Tangent splats (probe k) of the splats listed for one tile, in list order.
std::vector<Splat<Dual>> tile_tangents(const View& V, const std::vector<int>& list, const double* P, long pitch,
                                       int deg, uint64_t seed, int64_t t, int k, long n) {
  int rows = n_rows(deg);
  std::vector<Splat<Dual>> out(list.size());
  std::vector<double> tan(rows);
  for (size_t q = 0; q < list.size(); ++q) {
    long i = list[q];
    for (int r = 0; r < rows; ++r) tan[r] = rademacher(seed, t, k, probe_entry(i, r, rows));
    out[q] = project(load_gaussian<Dual>(P, pitch, i, deg, tan.data()), V.cam);
  }
  return out;
}

// Sampled pixels of one view (coordinates xs, ys): colour (npix x 3), final T,
// n_contrib, the decision margin and n_contrib range as in or_render, and, if
// nu > 0, the image tangents J z_k (npix x nu x 3) for the probes of (seed, t).
// With n_leaves given, also the outcomes of BlendOutcomes (at most max_leaves
// per pixel, flips with bounds up to branch_min summed instead): their count
// (-1 when there are more), colour (npix x max_leaves x 3), final T (npix x
// max_leaves), image tangents (npix x max_leaves x nu x 3, if nu > 0) and the
// sums rest / t_rest.
void or_render_pixels(const double* P, long pitch, long n, int deg, const double* cam24, int tw, int th, long npix,
                      const int32_t* xs, const int32_t* ys, uint64_t seed, int64_t t, int nu, double* rgb,
                      double* T_out, int32_t* nc_out, double* margin, double* jz, int32_t* nc_range,
                      double* impact, double* t_impact, int32_t* flip_kinds, int max_leaves, double branch_min,
                      int32_t* n_leaves, double* leaf_rgb, double* leaf_T, double* leaf_jz, double* rest,
                      double* t_rest) {
  View V = build_view(P, pitch, n, deg, cam24, tw, th);
  std::vector<int> local;
  for (long q = 0; q < npix; ++q) {
    int x = xs[q], y = ys[q], tx = x / tw, ty = y / th;
    const std::vector<int>& list = V.lists[(size_t)ty * V.Tx + tx];
    double C[3], T, mg;
    int nc;
    blend(list, V.sp, x + 0.5, y + 0.5, C, T, nc, &mg, nullptr);
    for (int ch = 0; ch < 3; ++ch) rgb[3 * q + ch] = C[ch];
    T_out[q] = T;
    nc_out[q] = nc;
    int lo = nc, hi = nc;
    margin[q] = std::min(mg, binning_margin(V, tx, ty, x + 0.5, y + 0.5, nc, &lo, &hi));
    if (impact) {
      const Flip fl = blend_flips(V, (size_t)ty * V.Tx + tx, x + 0.5, y + 0.5, nc);
      impact[q] = fl.impact;
      if (t_impact) t_impact[q] = fl.t_impact;
      if (flip_kinds) flip_kinds[q] = fl.kinds;
      lo = fl.nc_lo;
      hi = fl.nc_hi;
    }
    if (nc_range) {
      nc_range[2 * q] = lo;
      nc_range[2 * q + 1] = hi;
    }
    if (n_leaves) {
      BlendOutcomes bo(V, (size_t)ty * V.Tx + tx, x + 0.5, y + 0.5, branch_min, (size_t)max_leaves);
      bo.walk(0, {}, 1.0, 0.0, 0.0, 0.0, 0.0, false);
      n_leaves[q] = bo.overflow ? -1 : (int)bo.leaves.size();
      rest[q] = bo.rest;
      t_rest[q] = bo.t_rest;
      if (!bo.overflow) {
        const int rows = n_rows(deg);
        for (size_t l = 0; l < bo.leaves.size(); ++l) {
          double C[3], T;
          blend_sequence<double>(bo.leaves[l], [&](int i) -> const Splat<double>& { return V.sp[i]; }, x + 0.5,
                                 y + 0.5, C, T);
          for (int ch = 0; ch < 3; ++ch) leaf_rgb[((size_t)q * max_leaves + l) * 3 + ch] = C[ch];
          leaf_T[(size_t)q * max_leaves + l] = T;
        }
        std::vector<double> tan(rows);
        for (int k = 0; k < nu; ++k) {
          std::map<int, Splat<Dual>> sd;  // the splats of the leaves, forward mode along probe k
          auto get = [&](int i) -> const Splat<Dual>& {
            auto it = sd.find(i);
            if (it != sd.end()) return it->second;
            for (int r = 0; r < rows; ++r) tan[r] = rademacher(seed, t, k, probe_entry(i, r, rows));
            return sd.emplace(i, project(load_gaussian<Dual>(P, pitch, i, deg, tan.data()), V.cam)).first->second;
          };
          for (size_t l = 0; l < bo.leaves.size(); ++l) {
            Dual Cd[3], Td;
            blend_sequence<Dual>(bo.leaves[l], get, x + 0.5, y + 0.5, Cd, Td);
            for (int ch = 0; ch < 3; ++ch) leaf_jz[(((size_t)q * max_leaves + l) * nu + k) * 3 + ch] = Cd[ch].d;
          }
        }
      }
    }
    if (nu > 0) {
      local.resize(list.size());
      for (size_t u = 0; u < list.size(); ++u) local[u] = (int)u;
      for (int k = 0; k < nu; ++k) {
        std::vector<Splat<Dual>> sd = tile_tangents(V, list, P, pitch, deg, seed, t, k, n);
        Dual Cd[3], Td;
        int ncd;
        blend(local, sd, x + 0.5, y + 0.5, Cd, Td, ncd, nullptr, nullptr);
        for (int ch = 0; ch < 3; ++ch) jz[(q * nu + k) * 3 + ch] = Cd[ch].d;
      }
    }
  }
}

// Gradient and Hutchinson rows (ns x rows each) of the sampled Gaussians of a
// full frame of views, as or_backward would give for them: only pixels of the
// tiles a Gaussian is listed in involve it.  flag[s] collects the reasons an
// FP32 evaluation may legitimately take another discrete decision somewhere in
// the sample's footprint: 1 its own tile set is within rounding of changing; at
// a pixel where it is visible, 2 its own alpha / cap / power decision is within
// the FP32 rounding bound of power_uncertainty, 4 the residual sign is within
// eps_img (the image tolerance) of flipping, 8 another splat's binning, 16
// another splat's threshold decision is within 1e-5 of flipping.
// grad_mass, hz_mass (ns x rows, may be null): the masses of the entries' sums
// (as or_backward).  hz_sens (ns x rows, may be null): how far the Hutchinson
// entries move, at most, when every residual moves by e, the FP32 rounding
// bound of its pixel's colour (Flip::err of blend_flips) or eps_img (the
// tolerance the images are held to), whichever is smaller: the L1 Gauss-Newton weight
// 1/(4 max(|r|, gn_floor)) then changes by a factor within e / max(|r|,
// gn_floor) wherever |r| + e exceeds the floor, and the bound is that relative
// change carried through the absolute terms (blend_reverse_abs,
// project_reverse_abs).
// grad_allow, hz_allow (ns x rows, may be null): how far the entries may move
// when a decision of the sample's own flips in FP32 at a pixel where it is
// visible (its 1/255 skip, its cap, its power sign, or its membership in the
// tile's list), or a residual sign flips there (gradient only, 2 |dL/dC|): at
// each such pixel, the absolute values of the terms the sample adds there with
// its alpha uncapped, carried through project_reverse_abs.  grad_round,
// hz_round (may be null): the rounding its terms carry everywhere under the
// model of trace_rounding, the same way.
void or_backward_sampled(const double* P, long pitch, long n, int deg, const double* cams, int n_views, int tw,
                         int th, const double* target, int loss_kind, double gn_floor, uint64_t seed, int64_t t,
                         int nu, long ns, const int64_t* samples, double* grad_out, double* hz_out, int32_t* flag,
                         double eps_img, double* grad_mass, double* hz_mass, double* hz_sens, double* grad_allow,
                         double* hz_allow, double* grad_round, double* hz_round) {
  int rows = n_rows(deg);
  double m = 0.0;
  for (int v = 0; v < n_views; ++v) {
    Cam c = make_cam(cams + 24 * v);
    m += 3.0 * c.W * c.H;
  }
  for (long k = 0; k < ns * rows; ++k) {
    grad_out[k] = 0.0;
    if (hz_out) hz_out[k] = 0.0;
    if (grad_mass) grad_mass[k] = 0.0;
    if (hz_mass) hz_mass[k] = 0.0;
    if (hz_sens) hz_sens[k] = 0.0;
    if (grad_allow) grad_allow[k] = 0.0;
    if (hz_allow) hz_allow[k] = 0.0;
    if (grad_round) grad_round[k] = 0.0;
    if (hz_round) hz_round[k] = 0.0;
  }
  const bool masses = grad_mass || hz_mass || hz_sens;
  const bool allow = grad_allow != nullptr;
  for (long sidx = 0; sidx < ns; ++sidx) flag[sidx] = 0;
  long img_off = 0;
  std::vector<double> g_acc(rows);
  for (int v = 0; v < n_views; ++v) {
    View V = build_view(P, pitch, n, deg, cams + 24 * v, tw, th);
    long HW = (long)V.cam.W * V.cam.H;
    const double* tg = target + img_off;
    // tiles that list a sampled Gaussian
    std::vector<char> need((size_t)V.Tx * V.Ty, 0);
    for (long sidx = 0; sidx < ns; ++sidx) {
      long i = samples[sidx];
      if (!V.sp[i].valid) continue;
      const int* h = &V.hi[4 * i];
      const int* l = &V.lo[4 * i];
      if (!(h[0] == l[0] && h[1] == l[1] && h[2] == l[2] && h[3] == l[3])) flag[sidx] |= 1;
      for (int ty = h[2]; ty < h[3]; ++ty)
        for (int tx = h[0]; tx < h[1]; ++tx) need[(size_t)ty * V.Tx + tx] = 1;
    }
    std::vector<std::vector<double>> cot(1 + nu, std::vector<double>((size_t)n * NQ, 0.0));
    // masses: 0 the gradient, 1..nu the probes, nu+1..2nu the probes' sensitivity
    std::vector<std::vector<double>> cab(masses ? 1 + 2 * nu : 0, std::vector<double>((size_t)n * NQ, 0.0));
    // allowances per sample and stream (0 the gradient, 1..nu the probes), NQ each
    std::vector<double> al(allow ? (size_t)ns * (1 + nu) * NQ : 0, 0.0);
    // the rounding of every splat's terms, per stream (n x NQ each)
    std::vector<std::vector<double>> cround(allow ? 1 + nu : 0, std::vector<double>((size_t)n * NQ, 0.0));
    TraceRounding trel;
    std::vector<OwnFlip> pflips;
    std::vector<double> cflipw(allow ? (size_t)n * NQ : 0, 0.0);  // dL/dC uncertainty, every splat
    struct Own {
      long sidx;
      double a, G, dx, dy, T;
      bool own;  // its own decision or its tile membership may flip here
    };
    std::vector<Own> owns;
    double own_cmax = 0.0;  // the largest colour channel of the current tile's splats
    auto own_add = [&](const Own& q, const double wv[3], double* out) {
      own_terms(V.sp[samples[q.sidx]], OwnFlip{(int)samples[q.sidx], q.a, q.G, q.dx, q.dy, q.T}, own_cmax, wv, out);
    };
    std::vector<int> local;
    for (int ty = 0; ty < V.Ty; ++ty)
      for (int tx = 0; tx < V.Tx; ++tx) {
        if (!need[(size_t)ty * V.Tx + tx]) continue;
        const std::vector<int>& list = V.lists[(size_t)ty * V.Tx + tx];
        const std::vector<int>& amb = V.amb[(size_t)ty * V.Tx + tx];
        own_cmax = V.tile_cmax[(size_t)ty * V.Tx + tx];
        std::vector<std::vector<Splat<Dual>>> sd(nu);
        for (int k = 0; k < nu; ++k) sd[k] = tile_tangents(V, list, P, pitch, deg, seed, t, k, n);
        local.resize(list.size());
        for (size_t u = 0; u < list.size(); ++u) local[u] = (int)u;
        for (int y = ty * th; y < std::min((ty + 1) * th, V.cam.H); ++y)
          for (int x = tx * tw; x < std::min((tx + 1) * tw, V.cam.W); ++x) {
            double C[3], T, mg;
            int nc;
            std::vector<Contrib> tr;
            blend(list, V.sp, x + 0.5, y + 0.5, C, T, nc, &mg, &tr);
            long px = (long)y * V.cam.W + x;
            double w[3], wgn[3], sens[3], rmin = kInf;
            pflips.clear();
            // the residual's uncertainty: the colour's rounding (capped at the
            // image tolerance) plus what decision flips do to it
            double e_px = 0.0;
            if (masses) {
              const Flip fl = blend_flips(V, (size_t)ty * V.Tx + tx, x + 0.5, y + 0.5, nc, &pflips);
              e_px = std::min(fl.err, eps_img) + fl.impact;
            }
            for (int ch = 0; ch < 3; ++ch) {
              double r = C[ch] - tg[ch * HW + px];
              rmin = std::min(rmin, std::fabs(r));
              if (loss_kind == 0) {
                w[ch] = (r > 0 ? 1.0 : (r < 0 ? -1.0 : 0.0)) / (2.0 * m);
                wgn[ch] = 1.0 / (4.0 * std::max(std::fabs(r), gn_floor)) / m;
                sens[ch] = std::fabs(r) + e_px > gn_floor ? e_px / std::max(std::fabs(r), gn_floor) : 0.0;
              } else {
                w[ch] = r / m;
                wgn[ch] = 1.0 / m;
                sens[ch] = 0.0;
              }
            }
            const double mb = binning_margin(V, tx, ty, x + 0.5, y + 0.5);
            // reasons a sample visible here may see another decision in FP32:
            // 2 its own alpha / cap / power decision within the rounding bound, 4
            // the residual sign, 8 another splat's binning, 16 another splat's
            // threshold decision within 1e-5
            owns.clear();
            for (long sidx = 0; sidx < ns; ++sidx) {
              const int si = (int)samples[sidx];
              const Splat<double>& g = V.sp[si];
              if (!g.valid) continue;
              double dx = g.mx - (x + 0.5), dy = g.my - (y + 0.5);
              double power = -0.5 * (g.A * dx * dx + g.C * dy * dy) - g.B * dx * dy;
              double oG = g.o * std::exp(std::min(power, 0.0));
              if (oG < 0.5 * kAlphaMin) continue;
              const double dp = power_uncertainty(g, dx, dy);
              const bool own_near = std::fabs(std::min(oG, kAlphaMax) / kAlphaMin - 1.0) <= dp + 2e-6 ||
                                    std::fabs(oG / kAlphaMax - 1.0) <= dp + 2e-6 || std::fabs(power) <= dp;
              const bool in_tile = std::find(list.begin(), list.end(), si) != list.end();
              const bool membership = std::find(amb.begin(), amb.end(), si) != amb.end();
              if (own_near) flag[sidx] |= 2;
              if (rmin < eps_img) flag[sidx] |= 4;
              if (mb < 1e-5) flag[sidx] |= 8;
              if (mg < 1e-5) flag[sidx] |= 16;
              if (!allow || (!in_tile && !membership)) continue;
              // transmittance in front of it: its own trace entry, else that of
              // the first blended splat behind it, else the final T
              const float dsi = (float)g.depth;
              double Ts = T;
              for (const Contrib& e : tr) {
                const float de = (float)V.sp[e.i].depth;
                if (e.i == si || de > dsi || (de == dsi && e.i > si)) {
                  Ts = e.T;
                  break;
                }
              }
              // a flip the walk records for it (its own decisions, a termination
              // in front of it that the GPU may take elsewhere)
              bool listed = false;
              for (const OwnFlip& pf : pflips) listed = listed || pf.i == si;
              owns.push_back({sidx, std::min(oG, 1.0 - 1e-6), oG / g.o, dx, dy, Ts, own_near || membership || listed});
            }
            blend_reverse(tr, V.sp, w, cot[0].data());
            if (masses) blend_reverse_abs(tr, V.sp, w, cab[0].data());
            if (allow) {
              // dL/dC's own uncertainty: (L1) a residual whose sign may flip
              // changes it by 2 |w|, (L2) w = r/m moves by e_px/m
              double wflip[3];
              for (int ch = 0; ch < 3; ++ch) {
                const double r = std::fabs(C[ch] - tg[ch * HW + px]);
                wflip[ch] = loss_kind == 0 ? (r < e_px ? 2.0 * w[ch] : 0.0) : e_px / m;
              }
              for (const Own& q : owns) {
                double* out = al.data() + ((size_t)q.sidx * (1 + nu)) * NQ;
                if (q.own) own_add(q, w, out);
              }
              blend_reverse_abs(tr, V.sp, wflip, cflipw.data());
              trel = trace_rounding(tr, V.sp, pflips, own_cmax);
              blend_reverse_abs(tr, V.sp, w, cround[0].data(), &trel);
            }
            for (int k = 0; k < nu; ++k) {
              Dual Cd[3], Td;
              int ncd;
              blend(local, sd[k], x + 0.5, y + 0.5, Cd, Td, ncd, nullptr, nullptr);
              double wk[3], ws[3];
              for (int ch = 0; ch < 3; ++ch) {
                wk[ch] = wgn[ch] * Cd[ch].d;
                ws[ch] = wk[ch] * sens[ch];
              }
              if (allow) {
                for (const Own& q : owns)
                  if (q.own) own_add(q, wk, al.data() + ((size_t)q.sidx * (1 + nu) + 1 + k) * NQ);
                blend_reverse_abs(tr, V.sp, wk, cround[1 + k].data(), &trel);
              }
              blend_reverse(tr, V.sp, wk, cot[1 + k].data());
              if (masses) {
                blend_reverse_abs(tr, V.sp, wk, cab[1 + k].data());
                blend_reverse_abs(tr, V.sp, ws, cab[1 + nu + k].data());
              }
            }
          }
      }
    for (long sidx = 0; sidx < ns; ++sidx) {
      long i = samples[sidx];
      if (!V.sp[i].valid) continue;
      for (int st = 0; st <= nu; ++st) {
        std::fill(g_acc.begin(), g_acc.end(), 0.0);
        project_reverse(P, pitch, i, deg, V.cam, cot[st].data() + i * NQ, g_acc);
        for (int r = 0; r < rows; ++r) {
          if (st == 0) grad_out[sidx * rows + r] += g_acc[r];
          else hz_out[sidx * rows + r] += rademacher(seed, t, st - 1, probe_entry(i, r, rows)) * g_acc[r] / nu;
        }
      }
      for (int st = 0; masses && st <= 2 * nu; ++st) {
        std::fill(g_acc.begin(), g_acc.end(), 0.0);
        project_reverse_abs(P, pitch, i, deg, V.cam, cab[st].data() + i * NQ, g_acc);
        double* out = st == 0 ? grad_mass : (st <= nu ? hz_mass : hz_sens);
        if (!out) continue;
        for (int r = 0; r < rows; ++r) out[sidx * rows + r] += g_acc[r] / (st == 0 ? 1.0 : nu);
      }
      for (int q = 0; allow && q < NQ; ++q) al[((size_t)sidx * (1 + nu)) * NQ + q] += cflipw[(size_t)i * NQ + q];
      for (int st = 0; allow && st <= nu; ++st) {
        std::fill(g_acc.begin(), g_acc.end(), 0.0);
        project_reverse_abs(P, pitch, i, deg, V.cam, al.data() + ((size_t)sidx * (1 + nu) + st) * NQ, g_acc);
        double* out = st == 0 ? grad_allow : hz_allow;
        if (out)
          for (int r = 0; r < rows; ++r) out[sidx * rows + r] += g_acc[r] / (st == 0 ? 1.0 : nu);
        std::fill(g_acc.begin(), g_acc.end(), 0.0);
        project_reverse_abs(P, pitch, i, deg, V.cam, cround[st].data() + (size_t)i * NQ, g_acc);
        out = st == 0 ? grad_round : hz_round;
        if (out)
          for (int r = 0; r < rows; ++r) out[sidx * rows + r] += g_acc[r] / (st == 0 ? 1.0 : nu);
      }
    }
    img_off += 3 * HW;
  }
}

double or_hellinger(const double* mu1, const double* S1, double Z1, const double* mu2, const double* S2,
                    double Z2) {
  return hellinger(mu1, S1, Z1, mu2, S2, Z2);
}

void or_rotation_beta(const double* q, const double* s, double* beta) { rotation_beta(q, s, beta); }

}  // extern "C"
