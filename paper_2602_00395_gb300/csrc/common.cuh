// Shared device helpers of the gs3dtr CUDA library (sm_103a).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <type_traits>

#include "gs3dtr.h"

namespace gs {

// ------------------------------------------------------------ constants
// Blend thresholds of the 3DGS rasteriser the paper builds on (Sec. 3.1).
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;
constexpr float kDilation = 0.3f;    // added to the 2-D covariance diagonal
constexpr float kSlopeClamp = 1.3f;  // image-plane slope limit, x half field of view
constexpr int kRowSH = 11;
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ULL;
constexpr int kMaxViews = 64;

// Real SH normalisations, sqrt((2l+1)/(4pi) (l-m)!/(l+m)!) times the fixed
// factor of each Cartesian polynomial (3DGS sign convention).
constexpr float kY0 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
constexpr float kY1 = 0.48860251190291992f;   // sqrt(3/(4pi))
constexpr float kY2a = 1.0925484305920792f;   // sqrt(15/pi)/2
constexpr float kY2b = 0.31539156525252005f;  // sqrt(5/pi)/4
constexpr float kY2c = 0.54627421529603959f;  // sqrt(15/pi)/4
constexpr float kY3a = 0.59004358992664352f;  // sqrt(35/(2pi))/4
constexpr float kY3b = 2.8906114426405538f;   // sqrt(105/pi)/2
constexpr float kY3c = 0.45704579946446572f;  // sqrt(21/(2pi))/4
constexpr float kY3d = 0.37317633259011540f;  // sqrt(7/pi)/4
constexpr float kY3e = 1.4453057213202769f;   // sqrt(105/pi)/4

inline __host__ __device__ int n_coeffs(int deg) { return (deg + 1) * (deg + 1); }
inline __host__ __device__ int n_rows(int deg) { return kRowSH + 3 * n_coeffs(deg); }

// ------------------------------------------------------------ RNG
// SplitMix64 (Steele, Lea & Flood 2014): Weyl increment, then the finaliser
// with shifts 30, 27, 31.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + kGolden;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
// Probe seed and step as the kernels receive them: the step is read from device
// memory when t_dev is set (a call captured in a CUDA graph), else it is t.
struct ProbeArg {
  uint64_t seed;
  int64_t t;
  const int64_t* t_dev;
};
inline ProbeArg probe_arg(const gs_probe* p) {
  ProbeArg a;
  a.seed = p ? p->seed : 0;
  a.t = p ? p->t : 0;
  a.t_dev = p ? p->t_device : nullptr;
  return a;
}
__device__ __forceinline__ int64_t probe_step(const ProbeArg& a) { return a.t_dev ? *a.t_dev : a.t; }

// The items of a batch (gs_batch_item) as one kernel argument, with the first
// block of each item's share of a launch (first_block[n_items] = the grid).
struct BatchArg {
  int n_items;
  int first_block[GS_BATCH_MAX + 1];
  const float* P[GS_BATCH_MAX];
  int n[GS_BATCH_MAX], n_pad[GS_BATCH_MAX];
  const gs_camera* cam[GS_BATCH_MAX];
  int64_t t[GS_BATCH_MAX];
  float* grad[GS_BATCH_MAX];
  float* hz[GS_BATCH_MAX];
  float* ge[GS_BATCH_MAX];
  float* de[GS_BATCH_MAX];
  float eps[GS_BATCH_MAX];
  int hvp[GS_BATCH_MAX];
};
// The item whose share of the launch holds block `blk`.
__device__ __forceinline__ int batch_item(const BatchArg& ba, int blk) {
  int b = 0;
  while (b + 1 < ba.n_items && blk >= ba.first_block[b + 1]) ++b;
  return b;
}
// Host: the batch argument of items[0..n_items), blocks_of(item) blocks each.
template <class F>
BatchArg batch_arg(const gs_batch_item* items, int n_items, F blocks_of) {
  BatchArg a{};
  a.n_items = n_items;
  a.first_block[0] = 0;
  for (int b = 0; b < n_items; ++b) {
    const gs_batch_item& it = items[b];
    a.P[b] = it.x.data;
    a.n[b] = it.x.n;
    a.n_pad[b] = it.x.n_pad;
    a.cam[b] = it.cam;
    a.t[b] = it.t;
    a.grad[b] = it.grad.data;
    a.hz[b] = it.hz.data;
    a.ge[b] = it.g_ema.data;
    a.de[b] = it.d_ema.data;
    a.eps[b] = it.eps;
    a.hvp[b] = it.hvp;
    a.first_block[b + 1] = a.first_block[b] + blocks_of(it);
  }
  return a;
}

// Signs of Rademacher probe k at step t for the rows [0, rows) of Gaussian i:
// bit r is set where entry j = i * rows + r is -1.  Entry j is bit j mod 64 of
// the hash of word j / 64 (64 entries per hash), so the rows of one Gaussian
// (rows <= 64) take one or two hashes.
__device__ __forceinline__ uint64_t probe_signs(uint64_t seed, int64_t t, int k, uint64_t i, int rows) {
  const uint64_t key = seed ^ ((uint64_t)t * kGolden) ^ ((uint64_t)k << 56);
  const uint64_t j0 = i * (uint64_t)rows, w0 = j0 >> 6;
  const int off = (int)(j0 & 63);
  uint64_t bits = splitmix64(key ^ w0) >> off;
  if (off + rows > 64) bits |= splitmix64(key ^ (w0 + 1)) << (64 - off);
  return rows >= 64 ? bits : (bits & ((1ull << rows) - 1ull));
}

// ------------------------------------------------ forward-mode dual numbers
// Value plus N tangents; used to push the Rademacher directions through the
// projection (the "forward-mode AD" half of the Hessian-vector product).
template <int N>
struct Dn {
  float v;
  float d[N];
};

template <class S>
struct is_dual : std::false_type {};
template <int N>
struct is_dual<Dn<N>> : std::true_type {};

__device__ __forceinline__ float val(float x) { return x; }
template <int N>
__device__ __forceinline__ float val(const Dn<N>& x) { return x.v; }

template <int N>
__device__ __forceinline__ Dn<N> cst(float v) {
  Dn<N> r;
  r.v = v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = 0.f;
  return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator+(const Dn<N>& a, const Dn<N>& b) {
  Dn<N> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator-(const Dn<N>& a, const Dn<N>& b) {
  Dn<N> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator-(const Dn<N>& a) {
  Dn<N> r;
  r.v = -a.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = -a.d[k];
  return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator*(const Dn<N>& a, const Dn<N>& b) {
  Dn<N> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator/(const Dn<N>& a, const Dn<N>& b) {
  Dn<N> r;
  float ib = 1.0f / b.v;
  r.v = a.v * ib;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
  return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator+(const Dn<N>& a, float b) {
  Dn<N> r = a;
  r.v += b;
  return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator+(float b, const Dn<N>& a) { return a + b; }
template <int N>
__device__ __forceinline__ Dn<N> operator-(const Dn<N>& a, float b) {
  Dn<N> r = a;
  r.v -= b;
  return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator-(float b, const Dn<N>& a) {
  Dn<N> r = -a;
  r.v += b;
  return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator*(const Dn<N>& a, float b) {
  Dn<N> r;
  r.v = a.v * b;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * b;
  return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator*(float b, const Dn<N>& a) { return a * b; }
template <int N>
__device__ __forceinline__ Dn<N> operator/(const Dn<N>& a, float b) { return a * (1.0f / b); }
template <int N>
__device__ __forceinline__ Dn<N> operator/(float a, const Dn<N>& b) { return cst<N>(a) / b; }

__device__ __forceinline__ float sexp(float x) { return expf(x); }
__device__ __forceinline__ float ssqrt(float x) { return sqrtf(x); }
template <int N>
__device__ __forceinline__ Dn<N> sexp(const Dn<N>& a) {
  Dn<N> r;
  r.v = expf(a.v);
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = r.v * a.d[k];
  return r;
}
template <int N>
__device__ __forceinline__ Dn<N> ssqrt(const Dn<N>& a) {
  Dn<N> r;
  r.v = sqrtf(a.v);
  float h = 0.5f / r.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * h;
  return r;
}

template <class S>
__device__ __forceinline__ S constant(float v) {
  if constexpr (is_dual<S>::value) {
    return cst<sizeof(S::d) / sizeof(float)>(v);
  } else {
    return v;
  }
}

// ------------------------------------------------------------ SH basis
// Real spherical harmonics up to degree DEG at unit direction (x, y, z).
template <int DEG, class S>
__device__ __forceinline__ void sh_basis(const S& x, const S& y, const S& z, S* Y) {
  Y[0] = constant<S>(kY0);
  if constexpr (DEG >= 1) {
    Y[1] = -kY1 * y;
    Y[2] = kY1 * z;
    Y[3] = -kY1 * x;
  }
  if constexpr (DEG >= 2) {
    S xx = x * x, yy = y * y, zz = z * z;
    Y[4] = kY2a * (x * y);
    Y[5] = -kY2a * (y * z);
    Y[6] = kY2b * (2.0f * zz - xx - yy);
    Y[7] = -kY2a * (x * z);
    Y[8] = kY2c * (xx - yy);
    if constexpr (DEG >= 3) {
      Y[9] = -kY3a * y * (3.0f * xx - yy);
      Y[10] = kY3b * (x * y * z);
      Y[11] = -kY3c * y * (4.0f * zz - xx - yy);
      Y[12] = kY3d * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
      Y[13] = -kY3c * x * (4.0f * zz - xx - yy);
      Y[14] = kY3e * z * (xx - yy);
      Y[15] = -kY3a * x * (xx - 3.0f * yy);
    }
  }
}

// sum_k w_k grad Y_k at (x, y, z), treating x, y, z as independent.
template <int DEG>
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, const float* w, float g[3]) {
  g[0] = g[1] = g[2] = 0.f;
  if constexpr (DEG >= 1) {
    g[1] += -kY1 * w[1];
    g[2] += kY1 * w[2];
    g[0] += -kY1 * w[3];
  }
  if constexpr (DEG >= 2) {
    g[0] += kY2a * y * w[4];
    g[1] += kY2a * x * w[4];
    g[1] += -kY2a * z * w[5];
    g[2] += -kY2a * y * w[5];
    g[0] += -2.f * kY2b * x * w[6];
    g[1] += -2.f * kY2b * y * w[6];
    g[2] += 4.f * kY2b * z * w[6];
    g[0] += -kY2a * z * w[7];
    g[2] += -kY2a * x * w[7];
    g[0] += 2.f * kY2c * x * w[8];
    g[1] += -2.f * kY2c * y * w[8];
    if constexpr (DEG >= 3) {
      float xx = x * x, yy = y * y, zz = z * z;
      g[0] += -6.f * kY3a * x * y * w[9];
      g[1] += -kY3a * (3.f * xx - 3.f * yy) * w[9];
      g[0] += kY3b * y * z * w[10];
      g[1] += kY3b * x * z * w[10];
      g[2] += kY3b * x * y * w[10];
      g[0] += 2.f * kY3c * x * y * w[11];
      g[1] += -kY3c * (4.f * zz - xx - 3.f * yy) * w[11];
      g[2] += -8.f * kY3c * y * z * w[11];
      g[0] += -6.f * kY3d * x * z * w[12];
      g[1] += -6.f * kY3d * y * z * w[12];
      g[2] += kY3d * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
      g[0] += -kY3c * (4.f * zz - 3.f * xx - yy) * w[13];
      g[1] += 2.f * kY3c * x * y * w[13];
      g[2] += -8.f * kY3c * x * z * w[13];
      g[0] += 2.f * kY3e * x * z * w[14];
      g[1] += -2.f * kY3e * y * z * w[14];
      g[2] += kY3e * (xx - yy) * w[14];
      g[0] += -kY3a * (3.f * xx - 3.f * yy) * w[15];
      g[1] += 6.f * kY3a * x * y * w[15];
    }
  }
}

// ------------------------------------------------------ footprint extents
// Half-extents of the bounding box of a splat's alpha >= 1/255 footprint, kept
// in the last word of its record; binning narrows the splat's tile square to
// this box and the rasteriser tests its 8 x 8 pixel blocks against it.
// The footprint is the ellipse d^T Q d <= tau, tau = 2 ln(255 o), Q = [[A, B],
// [B, C]] the conic; its box has half-widths sqrt(tau C / det) and
// sqrt(tau A / det).  They are widened by 0.1% + 0.01 px, so that no pair an
// FP32 pixel test keeps falls outside, rounded up to half precision and packed
// (x in the low 16 bits, y in the high).  tau <= 0 (no pixel can reach 1/255)
// gives -inf, a non-finite half-width +inf.
__device__ __forceinline__ uint32_t footprint_extents(float A, float B, float C, float o) {
  const float tau = 2.f * __logf(255.f * o);
  unsigned short hx, hy;
  if (!(tau > 0.f)) {
    hx = hy = 0xFC00u;  // -inf
  } else {
    const float det = A * C - B * B;
    const float ex = sqrtf(tau * C / det), ey = sqrtf(tau * A / det);
    if (!(ex < 1e30f) || !(ey < 1e30f)) {
      hx = hy = 0x7C00u;  // +inf
    } else {
      hx = __half_as_ushort(__float2half_ru(ex * 1.001f + 0.01f));
      hy = __half_as_ushort(__float2half_ru(ey * 1.001f + 0.01f));
    }
  }
  return (uint32_t)hx | ((uint32_t)hy << 16);
}

// ---------------------------------------------------------- tile rectangle
// [x0, x1) x [y0, y1) of a splat, decided in FP32 with one rounding per step.
// The 3DGS square of half-width r:
//   x0 = clamp(floor((mx - r)/tw), 0, Tx),  x1 = clamp(floor((mx + (r + tw - 1))/tw), 0, Tx),
// intersected with the tiles the footprint box [mx - hx, mx + hx] reaches:
//   x0 >= floor((mx - hx)/tw),  x1 <= floor((mx + hx)/tw) + 1
// (the same for y; hx, hy the packed halves of `ext`).  A tile outside the box
// has no pixel centre where the splat's alpha reaches 1/255, so dropping it
// changes no image; -inf extents give an empty rectangle, +inf the square
// (binning passes +inf when the frame asks for the square alone).
__device__ __forceinline__ int clamp_floor(float f, int hi) {
  if (!(f > 0.0f)) return 0;  // NaN -> 0
  if (f > (float)hi) return hi;
  return (int)f;
}
__device__ __forceinline__ void tile_rect(float mx, float my, int r, uint32_t ext, int tw, int th, int Tx, int Ty,
                                          int& x0, int& x1, int& y0, int& y1) {
  const float hx = __half2float(__ushort_as_half((unsigned short)(ext & 0xffffu)));
  const float hy = __half2float(__ushort_as_half((unsigned short)(ext >> 16)));
  const float ftw = (float)tw, fth = (float)th;
  x0 = max(clamp_floor(floorf(__fdiv_rn(__fsub_rn(mx, (float)r), ftw)), Tx),
           clamp_floor(floorf(__fdiv_rn(__fsub_rn(mx, hx), ftw)), Tx));
  x1 = min(clamp_floor(floorf(__fdiv_rn(__fadd_rn(mx, (float)(r + tw - 1)), ftw)), Tx),
           clamp_floor(__fadd_rn(floorf(__fdiv_rn(__fadd_rn(mx, hx), ftw)), 1.0f), Tx));
  y0 = max(clamp_floor(floorf(__fdiv_rn(__fsub_rn(my, (float)r), fth)), Ty),
           clamp_floor(floorf(__fdiv_rn(__fsub_rn(my, hy), fth)), Ty));
  y1 = min(clamp_floor(floorf(__fdiv_rn(__fadd_rn(my, (float)(r + th - 1)), fth)), Ty),
           clamp_floor(__fadd_rn(floorf(__fdiv_rn(__fadd_rn(my, hy), fth)), 1.0f), Ty));
}

// ------------------------------------------------------- per-row tile spans
// Within the rectangle above, each tile row keeps only the tiles that the
// footprint ellipse reaches.  In units of the half-extents (u = dx/hx,
// v = dy/hy) the ellipse d^T Q d <= tau is u^2 - 2 rho u v + v^2 <= 1 - rho^2
// with rho = -B / sqrt(A C), because hx^2 = tau C/det, hy^2 = tau A/det and the
// off-diagonal of tau Q^-1 is rho hx hy.  Over the row's band of v the right
// end u = rho v + sqrt((1 - rho^2)(1 - v^2)) peaks at v = rho and the left end
// at v = -rho, so each is taken at that v clamped into the band.  The band is
// the tile row's full height; the ends are widened by 1 % of hx + 0.5 px, which
// covers the different rounding-up of hx and hy.  Every operation is one FP32
// rounding (the order is part of the binning rule).  Without finite positive
// extents (or with footprint_bins = 0) a row keeps the whole rectangle row.
struct FootRows {
  float mx, my, hx, hy, rho, q, mgn;
  int x0, x1, y0, y1;
  bool exact;
};

__device__ __forceinline__ FootRows foot_rows(float mx, float my, float A, float B, float C, int r, uint32_t ext,
                                              bool footprint, int tw, int th, int Tx, int Ty) {
  FootRows f;
  tile_rect(mx, my, r, footprint ? ext : 0x7C007C00u, tw, th, Tx, Ty, f.x0, f.x1, f.y0, f.y1);
  f.mx = mx;
  f.my = my;
  f.hx = __half2float(__ushort_as_half((unsigned short)(ext & 0xffffu)));
  f.hy = __half2float(__ushort_as_half((unsigned short)(ext >> 16)));
  f.exact = footprint && f.hx > 0.f && f.hy > 0.f && f.hx < 65536.f && f.hy < 65536.f && A > 0.f && C > 0.f;
  float rho = __fdiv_rn(-B, __fsqrt_rn(__fmul_rn(A, C)));
  rho = fminf(fmaxf(rho, -1.f), 1.f);
  f.rho = f.exact ? rho : 0.f;
  f.q = fmaxf(0.f, __fsub_rn(1.f, __fmul_rn(f.rho, f.rho)));
  f.mgn = __fadd_rn(__fmul_rn(0.01f, f.hx), 0.5f);
  return f;
}

// v of the band edge at pixel row y.
__device__ __forceinline__ float band_v(const FootRows& f, int y) { return __fdiv_rn(__fsub_rn((float)y, f.my), f.hy); }

// Tiles [a, b) of tile row ty, given the v of its band's edges (band_v at ty th
// and (ty + 1) th; a row's lower edge is the next row's upper edge, so the
// callers walk the rows computing each edge once).  tw is a power of two, so
// x / tw is the exact product by 1 / tw.
__device__ __forceinline__ void row_span_v(const FootRows& f, float vlo, float vhi, int tw, int Tx, int& a, int& b) {
  a = f.x0;
  b = f.x1;
  if (!f.exact) return;
  if (vhi < -1.f || vlo > 1.f) {
    b = a;
    return;
  }
  const float vr = fminf(fmaxf(f.rho, vlo), vhi);
  const float vl = fminf(fmaxf(-f.rho, vlo), vhi);
  const float sr = __fsqrt_rn(fmaxf(0.f, __fmul_rn(f.q, __fsub_rn(1.f, __fmul_rn(vr, vr)))));
  const float sl = __fsqrt_rn(fmaxf(0.f, __fmul_rn(f.q, __fsub_rn(1.f, __fmul_rn(vl, vl)))));
  const float xr = __fadd_rn(__fadd_rn(f.mx, __fmul_rn(f.hx, __fadd_rn(__fmul_rn(f.rho, vr), sr))), f.mgn);
  const float xl = __fsub_rn(__fadd_rn(f.mx, __fmul_rn(f.hx, __fsub_rn(__fmul_rn(f.rho, vl), sl))), f.mgn);
  const float itw = 1.0f / (float)tw;
  a = max(a, clamp_floor(floorf(__fmul_rn(xl, itw)), Tx));
  b = min(b, clamp_floor(__fadd_rn(floorf(__fmul_rn(xr, itw)), 1.0f), Tx));
  if (b < a) b = a;
}

// Number of (tile, splat) pairs of a splat.
__device__ __forceinline__ uint32_t foot_count(const FootRows& f, int tw, int th, int Tx) {
  if (f.x1 <= f.x0 || f.y1 <= f.y0) return 0;
  if (!f.exact) return (uint32_t)(f.x1 - f.x0) * (uint32_t)(f.y1 - f.y0);
  uint32_t n = 0;
  float vlo = band_v(f, f.y0 * th);
  for (int ty = f.y0; ty < f.y1; ++ty) {
    const float vhi = band_v(f, (ty + 1) * th);
    int a, b;
    row_span_v(f, vlo, vhi, tw, Tx, a, b);
    n += (uint32_t)(b - a);
    vlo = vhi;
  }
  return n;
}

// ------------------------------------------------- async copies (TMA bulk)
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// One non-multicast bulk copy global -> this CTA's shared memory, completing on bar.
// dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for phase `parity` of bar.  Returns false (and raises
// GS_FLAG_TIMEOUT) if the phase did not complete within the limit.
constexpr uint32_t kWaitLimit = 1u << 22;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int32_t* status) {
  for (uint32_t it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  if (status) atomicOr(status, GS_FLAG_TIMEOUT);
  return false;
}

// ---------------------------------------------------------- frames
// Tile shapes the kernels support: two pixels per thread and warps covering
// 8 x 8 pixel blocks, so tile_w is 8, 16 or 32, tile_h a power of two >= 8, and
// tile_w * tile_h is 64, 128, 256 or 512 (at most eight warps per tile).
inline bool frame_ok(gs_frame fr) {
  auto pow2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
  const int tt = fr.tile_w * fr.tile_h;
  return fr.n_views >= 1 && fr.width >= 1 && fr.height >= 1 && (fr.tile_w == 8 || fr.tile_w == 16 || fr.tile_w == 32) &&
         pow2(fr.tile_h) && fr.tile_h >= 8 && (tt == 64 || tt == 128 || tt == 256 || tt == 512) &&
         (fr.footprint_bins == 0 || fr.footprint_bins == 1) &&
         (fr.batch == 0 || (fr.batch % 32 == 0 && fr.batch >= 32 && fr.batch <= 512));
}

// ---------------------------------------------------------- host errors
void set_error(const char* fmt, ...);
gs_status check_launch(const char* what);

}  // namespace gs

#define GS_REQUIRE(cond, ...)          \
  do {                                 \
    if (!(cond)) {                     \
      gs::set_error(__VA_ARGS__);      \
      return GS_ERR_INVALID_ARG;       \
    }                                  \
  } while (0)
