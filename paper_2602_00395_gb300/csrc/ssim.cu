// gs_dssim_cotangents: the image-space vectors of the pixel loss
// (1 - lambda) L1 + lambda D-SSIM of Eq. pixel_loss (Sec. 3.2, D-SSIM = 1 - SSIM,
// m = 6 H W per view) for the reverse pass (GS_LOSS_COTANGENT):
//   stream 0   dL/dC = ((1 - lambda) sign(r) - lambda sum_p dS_p/dC) / (2m)
//   stream k   (1 - lambda)/(4 max(|r|, floor))/m . d_k + A[lambda/(4 max(1 - S, floor))/m . dS[d_k]]
// with d_k = J z_k the image tangents, dS[d] the directional derivative of the
// SSIM map and A its adjoint.  SSIM of one channel uses the 11 x 11 Gaussian
// window of standard deviation 1.5 (zeros outside the image), C1 = 0.01^2,
// C2 = 0.03^2.  As a function of the window means mx = G*x, Ex2 = G*(x^2),
// Exy = G*(x y) of the rendered channel x (the target's are constants):
//   A[a] = G*(a dS/dmx) + 2 x G*(a dS/dEx2) + y G*(a dS/dExy)   (G is symmetric)
//   dS[d] = dS/dmx G*d + dS/dEx2 G*(2 x d) + dS/dExy G*(y d)
//
// Every pass works on 32 x 32 output tiles of one (view, channel) plane: the
// inputs of the tile and its 5-pixel halo go to shared memory (zero outside
// the image), the products are filtered horizontally into shared memory, then
// vertically, and an epilogue combines the filtered values at each pixel.
#include <cmath>

#include "common.cuh"

namespace gs {
namespace {

constexpr int kR = 5, kTile = 32, kIn = kTile + 2 * kR;  // 42
constexpr int kSsimThreads = 256;
constexpr float kC1 = 1e-4f, kC2 = 9e-4f;
__constant__ float c_win[2 * kR + 1];

struct Plane {
  int W, H, planes;  // planes = views x 3
};

// inputs of the tile (with halo) of NIN planes into s_in[NIN][kIn][kIn]
template <int NIN>
__device__ __forceinline__ void load_tile(const float* const (&src)[NIN], size_t plane_off, int W, int H, int x0,
                                          int y0, float (*s_in)[kIn][kIn]) {
  for (int q = threadIdx.x; q < kIn * kIn; q += blockDim.x) {
    const int ty = q / kIn, tx = q - ty * kIn;
    const int gx = x0 - kR + tx, gy = y0 - kR + ty;
    const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
    const size_t at = plane_off + (size_t)(in ? gy : 0) * W + (in ? gx : 0);
#pragma unroll
    for (int k = 0; k < NIN; ++k) s_in[k][ty][tx] = in ? src[k][at] : 0.f;
  }
}

// Horizontal window sums of NOUT products (prod of the NIN inputs at (ty, tx))
// for all kIn rows and the kTile output columns.  A thread covers kCols adjacent
// columns of one row and reads each input value once; every sum still adds its
// 11 terms in window order.
constexpr int kCols = 4, kRows = 4;
template <int NIN, int NOUT, class Prod>
__device__ __forceinline__ void filter_tile(float (*s_in)[kIn][kIn], float (*s_h)[kIn][kTile], Prod prod) {
  for (int q = threadIdx.x; q < kIn * (kTile / kCols); q += blockDim.x) {
    const int ty = q / (kTile / kCols), ox0 = (q - ty * (kTile / kCols)) * kCols;
    float acc[NOUT][kCols];
#pragma unroll
    for (int o = 0; o < NOUT; ++o)
#pragma unroll
      for (int j = 0; j < kCols; ++j) acc[o][j] = 0.f;
#pragma unroll
    for (int c = 0; c < kCols + 2 * kR; ++c) {
      float v[NIN];
#pragma unroll
      for (int k = 0; k < NIN; ++k) v[k] = s_in[k][ty][ox0 + c];
      float p[NOUT];
      prod(v, p);
#pragma unroll
      for (int j = 0; j < kCols; ++j) {
        const int dd = c - j;
        if (dd >= 0 && dd <= 2 * kR) {
#pragma unroll
          for (int o = 0; o < NOUT; ++o) acc[o][j] += c_win[dd] * p[o];
        }
      }
    }
#pragma unroll
    for (int o = 0; o < NOUT; ++o)
#pragma unroll
      for (int j = 0; j < kCols; ++j) s_h[o][ty][ox0 + j] = acc[o][j];
  }
}

// Vertical window sums at output rows oy0 .. oy0 + kRows - 1 of column ox, each
// horizontal sum read once.
template <int NOUT>
__device__ __forceinline__ void vertical(float (*s_h)[kIn][kTile], int oy0, int ox, float (&out)[NOUT][kRows]) {
#pragma unroll
  for (int o = 0; o < NOUT; ++o)
#pragma unroll
    for (int j = 0; j < kRows; ++j) out[o][j] = 0.f;
#pragma unroll
  for (int c = 0; c < kRows + 2 * kR; ++c) {
#pragma unroll
    for (int o = 0; o < NOUT; ++o) {
      const float hv = s_h[o][oy0 + c][ox];
#pragma unroll
      for (int j = 0; j < kRows; ++j) {
        const int dd = c - j;
        if (dd >= 0 && dd <= 2 * kR) out[o][j] += c_win[dd] * hv;
      }
    }
  }
}

// The output pixels of a thread: rows oy0 .. oy0 + kRows - 1 of column ox.
__device__ __forceinline__ void out_block(int& oy0, int& ox) {
  ox = threadIdx.x % kTile;
  oy0 = (threadIdx.x / kTile) * kRows;
}
static_assert(kSsimThreads * kRows == kTile * kTile, "one block of kRows pixels per thread");

// SSIM and its partials by the raw window moments at one pixel
__device__ __forceinline__ void ssim_at(float mx, float my, float ex2, float ey2, float exy, float& S, float& dmx,
                                        float& dex2, float& dexy) {
  const float sx2 = ex2 - mx * mx, sy2 = ey2 - my * my, sxy = exy - mx * my;
  const float A1 = 2.f * mx * my + kC1, A2 = 2.f * sxy + kC2;
  const float B1 = mx * mx + my * my + kC1, B2 = sx2 + sy2 + kC2;
  const float iB = 1.f / (B1 * B2);
  S = A1 * A2 * iB;
  const float d_mx = 2.f * A2 * iB * (my - mx * A1 / B1);
  const float d_sx2 = -S / B2;
  const float d_sxy = 2.f * A1 * iB;
  dmx = d_mx - 2.f * mx * d_sx2 - my * d_sxy;
  dex2 = d_sx2;
  dexy = d_sxy;
}

// pass 1: S and its partials per pixel; the objective's sum
__global__ void __launch_bounds__(kSsimThreads) ssim_stats_kernel(const float* __restrict__ img,
                                                                  const float* __restrict__ tgt, Plane pl, float lambda,
                                                                  float inv_2m, float* __restrict__ S,
                                                                  float* __restrict__ P1, float* __restrict__ P2,
                                                                  float* __restrict__ P3, float* __restrict__ loss) {
  extern __shared__ __align__(16) float smem[];
  float(*s_in)[kIn][kIn] = reinterpret_cast<float(*)[kIn][kIn]>(smem);
  float(*s_h)[kIn][kTile] = reinterpret_cast<float(*)[kIn][kTile]>(smem + 2 * kIn * kIn);
  __shared__ float s_red[kSsimThreads / 32];
  const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile;
  const size_t off = (size_t)blockIdx.z * pl.W * pl.H;
  const float* src[2] = {img, tgt};
  load_tile<2>(src, off, pl.W, pl.H, x0, y0, s_in);
  __syncthreads();
  filter_tile<2, 5>(s_in, s_h, [](const float (&v)[2], float (&p)[5]) {
    p[0] = v[0];
    p[1] = v[1];
    p[2] = v[0] * v[0];
    p[3] = v[1] * v[1];
    p[4] = v[0] * v[1];
  });
  __syncthreads();
  float lsum = 0.f;
  int oy0, ox;
  out_block(oy0, ox);
  float fb[5][kRows];
  vertical<5>(s_h, oy0, ox, fb);
#pragma unroll
  for (int j = 0; j < kRows; ++j) {
    const int oy = oy0 + j;
    const int gx = x0 + ox, gy = y0 + oy;
    if (gx >= pl.W || gy >= pl.H) continue;
    float s, d1, d2, d3;
    ssim_at(fb[0][j], fb[1][j], fb[2][j], fb[3][j], fb[4][j], s, d1, d2, d3);
    const size_t at = off + (size_t)gy * pl.W + gx;
    S[at] = s;
    P1[at] = d1;
    P2[at] = d2;
    P3[at] = d3;
    const float r = s_in[0][oy + kR][ox + kR] - s_in[1][oy + kR][ox + kR];
    lsum += ((1.f - lambda) * fabsf(r) + lambda * (1.f - s)) * inv_2m;
  }
  if (loss) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.f;
      for (int w = 0; w < kSsimThreads / 32; ++w) t += s_red[w];
      atomicAdd(loss, t);
    }
  }
}

// pass 2, all NP probes of the step in one launch (the image, target, S and
// partials read once): a_k = lambda/(4 max(1 - S, floor))/m . dS[d_k]; the
// probes' planes are `stride` floats apart
template <int NP>
__global__ void __launch_bounds__(kSsimThreads) ssim_jvp_kernel(const float* __restrict__ d,
                                                                const float* __restrict__ img,
                                                                const float* __restrict__ tgt, Plane pl, size_t stride,
                                                                const float* __restrict__ S,
                                                                const float* __restrict__ P1,
                                                                const float* __restrict__ P2,
                                                                const float* __restrict__ P3, float wscale,
                                                                float floor_, float* __restrict__ a) {
  extern __shared__ __align__(16) float smem[];
  float(*s_in)[kIn][kIn] = reinterpret_cast<float(*)[kIn][kIn]>(smem);
  float(*s_h)[kIn][kTile] = reinterpret_cast<float(*)[kIn][kTile]>(smem + (NP + 2) * kIn * kIn);
  const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile;
  const size_t off = (size_t)blockIdx.z * pl.W * pl.H;
  const float* src[NP + 2];
#pragma unroll
  for (int k = 0; k < NP; ++k) src[k] = d + (size_t)k * stride;
  src[NP] = img;
  src[NP + 1] = tgt;
  load_tile<NP + 2>(src, off, pl.W, pl.H, x0, y0, s_in);
  __syncthreads();
  filter_tile<NP + 2, 3 * NP>(s_in, s_h, [](const float (&v)[NP + 2], float (&p)[3 * NP]) {
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      p[3 * k] = v[k];
      p[3 * k + 1] = 2.f * v[NP] * v[k];
      p[3 * k + 2] = v[NP + 1] * v[k];
    }
  });
  __syncthreads();
  int oy0, ox;
  out_block(oy0, ox);
  float fb[3 * NP][kRows];
  vertical<3 * NP>(s_h, oy0, ox, fb);
#pragma unroll
  for (int j = 0; j < kRows; ++j) {
    const int oy = oy0 + j;
    const int gx = x0 + ox, gy = y0 + oy;
    if (gx >= pl.W || gy >= pl.H) continue;
    const size_t at = off + (size_t)gy * pl.W + gx;
    const float p1 = P1[at], p2 = P2[at], p3 = P3[at];
    const float w = wscale / (4.f * fmaxf(1.f - S[at], floor_));
#pragma unroll
    for (int k = 0; k < NP; ++k)
      a[(size_t)k * stride + at] = w * (p1 * fb[3 * k][j] + p2 * fb[3 * k + 1][j] + p3 * fb[3 * k + 2][j]);
  }
}

// pass 3: the adjoint of NA weight planes a_k (NA = 0: one stream with weights
// all 1, the gradient) plus the L1 part, into NA (or 1) cotangent images; the
// planes of a, d and cot are `stride` floats apart
template <int NA>
__global__ void __launch_bounds__(kSsimThreads) ssim_vjp_kernel(const float* __restrict__ a,
                                                                const float* __restrict__ img,
                                                                const float* __restrict__ tgt, Plane pl, size_t stride,
                                                                const float* __restrict__ P1,
                                                                const float* __restrict__ P2,
                                                                const float* __restrict__ P3,
                                                                const float* __restrict__ d, float lambda,
                                                                float inv_m, float floor_, float* __restrict__ cot) {
  constexpr int NS = NA > 0 ? NA : 1;  // output streams
  constexpr int NIN = NA + 3;
  extern __shared__ __align__(16) float smem[];
  float(*s_in)[kIn][kIn] = reinterpret_cast<float(*)[kIn][kIn]>(smem);
  float(*s_h)[kIn][kTile] = reinterpret_cast<float(*)[kIn][kTile]>(smem + NIN * kIn * kIn);
  const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile;
  const size_t off = (size_t)blockIdx.z * pl.W * pl.H;
  const float* src[NIN];
#pragma unroll
  for (int k = 0; k < NA; ++k) src[k] = a + (size_t)k * stride;
  src[NA] = P1;
  src[NA + 1] = P2;
  src[NA + 2] = P3;
  load_tile<NIN>(src, off, pl.W, pl.H, x0, y0, s_in);
  __syncthreads();
  filter_tile<NIN, 3 * NS>(s_in, s_h, [](const float (&v)[NIN], float (&p)[3 * NS]) {
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const float wk = NA > 0 ? v[k] : 1.f;  // weights all 1: the products are the partials
      p[3 * k] = wk * v[NA];
      p[3 * k + 1] = wk * v[NA + 1];
      p[3 * k + 2] = wk * v[NA + 2];
    }
  });
  __syncthreads();
  int oy0, ox;
  out_block(oy0, ox);
  float fb[3 * NS][kRows];
  vertical<3 * NS>(s_h, oy0, ox, fb);
#pragma unroll
  for (int j = 0; j < kRows; ++j) {
    const int oy = oy0 + j;
    const int gx = x0 + ox, gy = y0 + oy;
    if (gx >= pl.W || gy >= pl.H) continue;
    const size_t at = off + (size_t)gy * pl.W + gx;
    const float x = img[at], y = tgt[at], r = x - y;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const float A = fb[3 * k][j] + 2.f * x * fb[3 * k + 1][j] + y * fb[3 * k + 2][j];
      if (NA == 0)
        cot[at] = 0.5f * inv_m * ((1.f - lambda) * (float)((r > 0.f) - (r < 0.f)) - lambda * A);
      else
        cot[(size_t)k * stride + at] =
            (1.f - lambda) * inv_m / (4.f * fmaxf(fabsf(r), floor_)) * d[(size_t)k * stride + at] + A;
    }
  }
}

size_t smem_bytes(int nin, int nout) { return sizeof(float) * ((size_t)nin * kIn * kIn + (size_t)nout * kIn * kTile); }

cudaError_t set_window() {
  static bool done = false;
  if (done) return cudaSuccess;
  double g[2 * kR + 1], s = 0.0;
  for (int i = -kR; i <= kR; ++i) s += g[i + kR] = std::exp(-(double)(i * i) / (2.0 * 1.5 * 1.5));
  float gf[2 * kR + 1];
  for (int i = 0; i <= 2 * kR; ++i) gf[i] = (float)(g[i] / s);
  cudaError_t e = cudaMemcpyToSymbol(c_win, gf, sizeof(gf));
  if (e == cudaSuccess) {
    e = cudaFuncSetAttribute((const void*)ssim_stats_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes(2, 5));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute((const void*)ssim_jvp_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem_bytes(3, 3));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute((const void*)ssim_jvp_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem_bytes(4, 6));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute((const void*)ssim_vjp_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem_bytes(3, 3));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute((const void*)ssim_vjp_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem_bytes(4, 3));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute((const void*)ssim_vjp_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem_bytes(5, 6));
  }
  done = e == cudaSuccess;
  return e;
}

}  // namespace
}  // namespace gs

extern "C" size_t gs_dssim_workspace_size(gs_frame frame, int32_t nu) {
  if (frame.n_views < 1 || frame.width < 1 || frame.height < 1 || nu < 0 || nu > 2) return 0;
  const size_t plane = (size_t)frame.n_views * 3 * frame.width * frame.height;
  return plane * sizeof(float) * (4 + (size_t)nu);  // S, three partials, one weight map per probe
}

extern "C" gs_status gs_dssim_cotangents(gs_frame frame, const float* image, const float* target,
                                         const float* image_tangent, int32_t nu, float lambda, float gn_floor,
                                         int32_t want_grad, float* cot, float* loss_out, void* workspace,
                                         size_t workspace_bytes, int32_t* status, void* stream) {
  using namespace gs;
  (void)status;
  GS_REQUIRE(image && target && cot, "gs_dssim_cotangents: null argument");
  GS_REQUIRE(frame.n_views >= 1 && frame.width >= 1 && frame.height >= 1, "gs_dssim_cotangents: bad frame");
  GS_REQUIRE(nu >= 0 && nu <= 2 && (nu == 0 || image_tangent), "gs_dssim_cotangents: bad nu=%d or no tangents", nu);
  GS_REQUIRE(want_grad || nu > 0, "gs_dssim_cotangents: nothing to compute");
  GS_REQUIRE(lambda >= 0.f && lambda <= 1.f && gn_floor > 0.f, "gs_dssim_cotangents: bad lambda or floor");
  const size_t need = gs_dssim_workspace_size(frame, nu);
  GS_REQUIRE(workspace && workspace_bytes >= need, "gs_dssim_cotangents: workspace needs %zu bytes, got %zu", need,
             workspace_bytes);
  if (set_window() != cudaSuccess) return check_launch("gs_dssim_cotangents: window");
  cudaStream_t st = (cudaStream_t)stream;
  const Plane pl{frame.width, frame.height, frame.n_views * 3};
  const size_t plane = (size_t)pl.planes * pl.W * pl.H;
  float* ws = (float*)workspace;
  float *S = ws, *P1 = ws + plane, *P2 = ws + 2 * plane, *P3 = ws + 3 * plane, *A = ws + 4 * plane;
  const double m = 6.0 * frame.width * frame.height * frame.n_views;
  const float inv_m = (float)(1.0 / m), inv_2m = (float)(0.5 / m);
  const dim3 grid((pl.W + kTile - 1) / kTile, (pl.H + kTile - 1) / kTile, pl.planes);
  ssim_stats_kernel<<<grid, kSsimThreads, smem_bytes(2, 5), st>>>(image, target, pl, lambda, inv_2m, S, P1, P2, P3,
                                                                   loss_out);
  if (nu == 1)
    ssim_jvp_kernel<1><<<grid, kSsimThreads, smem_bytes(3, 3), st>>>(image_tangent, image, target, pl, plane, S, P1,
                                                                      P2, P3, lambda * inv_m, gn_floor, A);
  else if (nu == 2)
    ssim_jvp_kernel<2><<<grid, kSsimThreads, smem_bytes(4, 6), st>>>(image_tangent, image, target, pl, plane, S, P1,
                                                                      P2, P3, lambda * inv_m, gn_floor, A);
  float* cot_p = cot;
  if (want_grad) {
    ssim_vjp_kernel<0><<<grid, kSsimThreads, smem_bytes(3, 3), st>>>(nullptr, image, target, pl, plane, P1, P2, P3,
                                                                      nullptr, lambda, inv_m, gn_floor, cot_p);
    cot_p += plane;
  }
  if (nu == 1)
    ssim_vjp_kernel<1><<<grid, kSsimThreads, smem_bytes(4, 3), st>>>(A, image, target, pl, plane, P1, P2, P3,
                                                                      image_tangent, lambda, inv_m, gn_floor, cot_p);
  else if (nu == 2)
    ssim_vjp_kernel<2><<<grid, kSsimThreads, smem_bytes(5, 6), st>>>(A, image, target, pl, plane, P1, P2, P3,
                                                                      image_tangent, lambda, inv_m, gn_floor, cot_p);
  return check_launch("gs_dssim_cotangents");
}
