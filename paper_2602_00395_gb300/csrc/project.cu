// gs_project: EWA projection of every Gaussian into every view (Sec. 3.1 of
// arXiv 2602.00395, which defers the projection to 3DGS), optionally with the
// forward-mode tangents along the Rademacher probes of the Hutchinson estimator
// (Sec. 4.1; the paper adds forward-mode AD to the rasteriser, Sec. 5).
//
// One thread per Gaussian loops over the views, so each parameter column is read
// from HBM once per call and the probe signs are hashed once per call.  Output
// records are 48-byte AoS rows so that the rasteriser can move each one into
// shared memory with a single bulk copy.
#include "common.cuh"

namespace gs {
namespace {

template <class S>
__device__ __forceinline__ S clamp_const(const S& x, float lo, float hi, bool& clamped) {
  float v = val(x);
  clamped = (v < lo) || (v > hi);
  if (v < lo) return constant<S>(lo);
  if (v > hi) return constant<S>(hi);
  return x;
}

__device__ __forceinline__ void store_culled(float4* rec, size_t at) {
  rec[3 * at + 0] = make_float4(0.f, 0.f, 0.f, 0.f);
  rec[3 * at + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
  rec[3 * at + 2] = make_float4(0.f, 0.f, __int_as_float(0), 0.f);
}

// Minimum resident CTAs per SM requested for the projection (0: none).
#ifndef GS_PROJ_MIN_BLOCKS
#define GS_PROJ_MIN_BLOCKS 4
#endif
#if GS_PROJ_MIN_BLOCKS > 0
#define GS_PROJ_BOUNDS __launch_bounds__(128, GS_PROJ_MIN_BLOCKS)
#else
#define GS_PROJ_BOUNDS __launch_bounds__(128)
#endif

// Column i of the parameter matrix P (n Gaussians, row pitch n_pad) projected
// into views cams[0..V): record v * pitch + i of rec, tangent records
// (v * pitch + i) * (NU + 1) + 1 + k of tan, after a copy of the record at
// (v * pitch + i) * (NU + 1); columns n <= i < pitch are written culled.
// Called by every thread of a 128-thread block (the SH staging is block-wide).
template <int DEG, int NU>
__device__ __forceinline__ void project_column(const float* __restrict__ P, int n, int n_pad, int i, int pitch,
                                               const gs_camera* __restrict__ cams, int V, gs_frame fr, ProbeArg pa,
                                               float4* __restrict__ rec, float4* __restrict__ tan) {
  using S = typename std::conditional<NU == 0, float, Dn<(NU > 0 ? NU : 1)>>::type;
  constexpr int K = (DEG + 1) * (DEG + 1);
  constexpr int ROWS = kRowSH + 3 * K;
  // the block's SH coefficients, staged once and read per view from shared
  // memory (volatile: re-read, not held in registers across the view loop)
  __shared__ float s_sh[3 * K][128];
  for (int r = 0; r < 3 * K; ++r) s_sh[r][threadIdx.x] = i < n ? P[(size_t)(kRowSH + r) * n_pad + i] : 0.f;
  __syncthreads();
  const volatile float* vsh = &s_sh[0][0];
  if (i >= pitch) return;
  if (i >= n) {
    for (int v = 0; v < V; ++v) {
      store_culled(rec, (size_t)v * pitch + i);
      if (NU > 0)  // the record's copy and its tangents; no tangent array without probes
        for (int k = 0; k <= NU; ++k) store_culled(tan, ((size_t)v * pitch + i) * (NU + 1) + k);
    }
    return;
  }

  // probe signs: bit r of neg[k] is set where probe k is -1 on row r
  const uint64_t seed = pa.seed;
  const int64_t step = NU > 0 ? probe_step(pa) : 0;
  uint64_t neg[NU > 0 ? NU : 1];
#pragma unroll
  for (int k = 0; k < NU; ++k) neg[k] = probe_signs(seed, step, k, (uint64_t)i, ROWS);
  auto ld = [&](int r) -> S {
    float v = __ldg(P + (size_t)r * n_pad + i);
    if constexpr (NU == 0) {
      return v;
    } else {
      S s;
      s.v = v;
#pragma unroll
      for (int k = 0; k < NU; ++k) s.d[k] = ((neg[k] >> r) & 1ull) ? -1.f : 1.f;
      return s;
    }
  };

  const S mu0 = ld(0), mu1 = ld(1), mu2 = ld(2);
  // rotation of the normalised quaternion (x, y, z, w)
  S qx = ld(6), qy = ld(7), qz = ld(8), qw = ld(9);
  {
    S r = ssqrt(qx * qx + qy * qy + qz * qz + qw * qw);
    qx = qx / r; qy = qy / r; qz = qz / r; qw = qw / r;
  }
  S R[3][3];
  R[0][0] = 1.f - 2.f * (qy * qy + qz * qz);
  R[0][1] = 2.f * (qx * qy - qw * qz);
  R[0][2] = 2.f * (qx * qz + qw * qy);
  R[1][0] = 2.f * (qx * qy + qw * qz);
  R[1][1] = 1.f - 2.f * (qz * qz + qx * qx);
  R[1][2] = 2.f * (qy * qz - qw * qx);
  R[2][0] = 2.f * (qx * qz - qw * qy);
  R[2][1] = 2.f * (qy * qz + qw * qx);
  R[2][2] = 1.f - 2.f * (qx * qx + qy * qy);
  S s2[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) s2[a] = sexp(2.f * ld(3 + a));
  // Sigma = R diag(s^2) R^T (upper triangle)
  S Sg[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = a; b < 3; ++b) Sg[a][b] = R[a][0] * s2[0] * R[b][0] + R[a][1] * s2[1] * R[b][1] + R[a][2] * s2[2] * R[b][2];
  Sg[1][0] = Sg[0][1];
  Sg[2][0] = Sg[0][2];
  Sg[2][1] = Sg[1][2];
  const S opac = 1.f / (1.f + sexp(-ld(10)));

#pragma unroll 1
  for (int v = 0; v < V; ++v) {
    const gs_camera* c = cams + v;
    const size_t at = (size_t)v * pitch + i;
    float Rc[3][3], tc[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
      for (int b = 0; b < 3; ++b) Rc[a][b] = c->viewmat[4 * a + b];
      tc[a] = c->viewmat[4 * a + 3];
    }
    const float fx = c->fx, fy = c->fy;
    S t0 = Rc[0][0] * mu0 + Rc[0][1] * mu1 + Rc[0][2] * mu2 + tc[0];
    S t1 = Rc[1][0] * mu0 + Rc[1][1] * mu1 + Rc[1][2] * mu2 + tc[1];
    S t2 = Rc[2][0] * mu0 + Rc[2][1] * mu1 + Rc[2][2] * mu2 + tc[2];
    if (!(val(t2) > c->near_plane)) {
      store_culled(rec, at);
      if (NU > 0)  // the record's copy and its tangents; no tangent array without probes
        for (int k = 0; k <= NU; ++k) store_culled(tan, ((size_t)v * pitch + i) * (NU + 1) + k);
      continue;
    }
    // camera-frame covariance Rc Sigma Rc^T
    S Sc[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      S tmp[3];
#pragma unroll
      for (int b = 0; b < 3; ++b) tmp[b] = Rc[a][0] * Sg[0][b] + Rc[a][1] * Sg[1][b] + Rc[a][2] * Sg[2][b];
#pragma unroll
      for (int b = a; b < 3; ++b) Sc[a][b] = tmp[0] * Rc[b][0] + tmp[1] * Rc[b][1] + tmp[2] * Rc[b][2];
    }
    const float limx = kSlopeClamp * 0.5f * (float)fr.width / fx;
    const float limy = kSlopeClamp * 0.5f * (float)fr.height / fy;
    const S u = t0 / t2, w_ = t1 / t2;
    bool clx, cly;
    const S uc = clamp_const(u, -limx, limx, clx);
    const S vc = clamp_const(w_, -limy, limy, cly);
    const S J00 = fx / t2, J02 = -fx * uc / t2;
    const S J11 = fy / t2, J12 = -fy * vc / t2;
    const S a = J00 * J00 * Sc[0][0] + 2.f * J00 * J02 * Sc[0][2] + J02 * J02 * Sc[2][2] + kDilation;
    const S b = J00 * J11 * Sc[0][1] + J00 * J12 * Sc[0][2] + J02 * J11 * Sc[1][2] + J02 * J12 * Sc[2][2];
    const S cc = J11 * J11 * Sc[1][1] + 2.f * J11 * J12 * Sc[1][2] + J12 * J12 * Sc[2][2] + kDilation;
    const S det = a * cc - b * b;
    if (!(val(det) > 0.f)) {
      store_culled(rec, at);
      if (NU > 0)  // the record's copy and its tangents; no tangent array without probes
        for (int k = 0; k <= NU; ++k) store_culled(tan, ((size_t)v * pitch + i) * (NU + 1) + k);
      continue;
    }
    const S idet = 1.f / det;
    const S cA = cc * idet, cB = -b * idet, cC = a * idet;
    const float mid = 0.5f * (val(a) + val(cc));
    const float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - val(det)));
    const int radius = (int)ceilf(3.f * sqrtf(lam));
    const S mx = fx * u + c->cx, my = fy * w_ + c->cy;

    // view-dependent colour
    float cp[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) cp[q] = -(Rc[0][q] * tc[0] + Rc[1][q] * tc[1] + Rc[2][q] * tc[2]);
    S d0 = mu0 - cp[0], d1 = mu1 - cp[1], d2 = mu2 - cp[2];
    const S dn = ssqrt(d0 * d0 + d1 * d1 + d2 * d2);
    d0 = d0 / dn; d1 = d1 / dn; d2 = d2 / dn;
    S Y[K];
    sh_basis<DEG>(d0, d1, d2, Y);
    // rgb = 0.5 + sum_k Y_k sh_k; the coefficients are plain parameters whose
    // probe tangents are the signs z, read per view from the staged copy
    S rgb[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      S acc = constant<S>(0.5f);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int row = kRowSH + 3 * k + ch;
        const float sh = vsh[(3 * k + ch) * 128 + threadIdx.x];
        if constexpr (NU == 0) {
          acc = acc + Y[k] * sh;
        } else {
          acc.v += Y[k].v * sh;
#pragma unroll
          for (int p = 0; p < NU; ++p)
            acc.d[p] += Y[k].d[p] * sh + (((neg[p] >> row) & 1ull) ? -Y[k].v : Y[k].v);
        }
      }
      rgb[ch] = (val(acc) < 0.f) ? constant<S>(0.f) : acc;
    }

    rec[3 * at + 0] = make_float4(val(mx), val(my), val(cA), val(cB));
    rec[3 * at + 1] = make_float4(val(cC), val(opac), val(rgb[0]), val(rgb[1]));
    rec[3 * at + 2] = make_float4(val(rgb[2]), val(t2), __int_as_float(radius),
                                  __uint_as_float(footprint_extents(val(cA), val(cB), val(cC), val(opac))));
    if constexpr (NU > 0) {
      // the record again, in front of its tangent records: the forward blend
      // stages all of a splat's records with one copy
      const size_t t0 = ((size_t)v * pitch + i) * (NU + 1);
      tan[3 * t0 + 0] = rec[3 * at + 0];
      tan[3 * t0 + 1] = rec[3 * at + 1];
      tan[3 * t0 + 2] = rec[3 * at + 2];
#pragma unroll
      for (int k = 0; k < NU; ++k) {
        const size_t tk = ((size_t)v * pitch + i) * (NU + 1) + 1 + k;
        tan[3 * tk + 0] = make_float4(mx.d[k], my.d[k], cA.d[k], cB.d[k]);
        tan[3 * tk + 1] = make_float4(cC.d[k], opac.d[k], rgb[0].d[k], rgb[1].d[k]);
        tan[3 * tk + 2] = make_float4(rgb[2].d[k], 0.f, 0.f, 0.f);
      }
    }
    (void)clx;
    (void)cly;
  }
}

template <int DEG, int NU>
__global__ void GS_PROJ_BOUNDS project_kernel(const float* __restrict__ P, int n, int n_pad,
                                              const gs_camera* __restrict__ cams, gs_frame fr, ProbeArg pa,
                                              float4* __restrict__ rec, float4* __restrict__ tan) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  project_column<DEG, NU>(P, n, n_pad, i, n_pad, cams, fr.n_views, fr, pa, rec, tan);
}

// A batch: item b's share of the grid projects its columns into its camera,
// records in slot b (pitch n_pad_max) with its own probe step.
template <int DEG, int NU>
__global__ void GS_PROJ_BOUNDS project_batch_kernel(BatchArg ba, int pitch, gs_frame fr, ProbeArg pa,
                                                    float4* __restrict__ rec, float4* __restrict__ tan) {
  const int b = batch_item(ba, (int)blockIdx.x);
  const int i = ((int)blockIdx.x - ba.first_block[b]) * blockDim.x + threadIdx.x;
  pa.t = ba.t[b];
  pa.t_dev = nullptr;
  project_column<DEG, NU>(ba.P[b], ba.n[b], ba.n_pad[b], i, pitch, ba.cam[b], 1, fr, pa,
                          rec + 3 * (size_t)b * pitch, tan ? tan + 3 * (size_t)b * (NU + 1) * pitch : nullptr);
}

template <int DEG, int NU>
void launch_project(const gs_params* x, const gs_camera* cams, gs_frame fr, ProbeArg pa, gs_projected* out,
                    cudaStream_t st) {
  const int threads = 128;  // the kernel's shared staging is sized for 128 threads
  const int blocks = (x->n_pad + threads - 1) / threads;
  project_kernel<DEG, NU><<<blocks, threads, 0, st>>>(x->data, x->n, x->n_pad, cams, fr, pa,
                                                      reinterpret_cast<float4*>(out->rec),
                                                      reinterpret_cast<float4*>(out->tangent));
}

template <int DEG>
void dispatch_nu(int nu, const gs_params* x, const gs_camera* cams, gs_frame fr, ProbeArg pa, gs_projected* out,
                 cudaStream_t st) {
  if (nu == 0) launch_project<DEG, 0>(x, cams, fr, pa, out, st);
  else if (nu == 1) launch_project<DEG, 1>(x, cams, fr, pa, out, st);
  else launch_project<DEG, 2>(x, cams, fr, pa, out, st);
}

}  // namespace
}  // namespace gs

extern "C" gs_status gs_project(const gs_params* x, const gs_camera* cams, gs_frame frame, const gs_probe* probe,
                                gs_projected* out, int32_t* status, void* stream) {
  (void)status;
  GS_REQUIRE(x && out && cams, "gs_project: null argument");
  GS_REQUIRE(x->data && out->rec, "gs_project: null device buffer");
  GS_REQUIRE(x->n >= 0 && x->n_pad >= x->n && x->n_pad % 4 == 0, "gs_project: bad n=%d n_pad=%d", x->n, x->n_pad);
  GS_REQUIRE(frame.n_views >= 1 && frame.width >= 1 && frame.height >= 1, "gs_project: bad frame");
  const int nu = probe ? probe->nu : 0;
  if (x->sh_degree < 0 || x->sh_degree > 3 || nu < 0 || nu > 2) {
    gs::set_error("gs_project: unsupported sh_degree=%d nu=%d", x->sh_degree, nu);
    return GS_ERR_UNSUPPORTED;
  }
  GS_REQUIRE(nu == 0 || out->tangent, "gs_project: probes given but out->tangent is NULL");
  if (x->n_pad == 0) return GS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const gs::ProbeArg pa = gs::probe_arg(probe);
  switch (x->sh_degree) {
    case 0: gs::dispatch_nu<0>(nu, x, cams, frame, pa, out, st); break;
    case 1: gs::dispatch_nu<1>(nu, x, cams, frame, pa, out, st); break;
    case 2: gs::dispatch_nu<2>(nu, x, cams, frame, pa, out, st); break;
    default: gs::dispatch_nu<3>(nu, x, cams, frame, pa, out, st); break;
  }
  return gs::check_launch("gs_project");
}

namespace gs {
namespace {
template <int DEG>
void dispatch_batch(int nu, const BatchArg& ba, int pitch, gs_frame fr, ProbeArg pa, gs_projected* out,
                    cudaStream_t st) {
  const int blocks = ba.first_block[ba.n_items];
  float4* rec = reinterpret_cast<float4*>(out->rec);
  float4* tan = reinterpret_cast<float4*>(out->tangent);
  if (nu == 0) project_batch_kernel<DEG, 0><<<blocks, 128, 0, st>>>(ba, pitch, fr, pa, rec, nullptr);
  else if (nu == 1) project_batch_kernel<DEG, 1><<<blocks, 128, 0, st>>>(ba, pitch, fr, pa, rec, tan);
  else project_batch_kernel<DEG, 2><<<blocks, 128, 0, st>>>(ba, pitch, fr, pa, rec, tan);
}
}  // namespace
}  // namespace gs

extern "C" gs_status gs_project_batch(const gs_batch_item* items, int32_t n_items, int32_t n_pad_max, gs_frame frame,
                                      const gs_probe* probe, gs_projected* out, int32_t* status, void* stream) {
  (void)status;
  GS_REQUIRE(items && out && out->rec, "gs_project_batch: null argument");
  GS_REQUIRE(n_items >= 1 && n_items <= GS_BATCH_MAX, "gs_project_batch: n_items=%d outside [1, %d]", n_items,
             GS_BATCH_MAX);
  GS_REQUIRE(frame.n_views == n_items && frame.width >= 1 && frame.height >= 1,
             "gs_project_batch: frame.n_views must equal n_items");
  GS_REQUIRE(n_pad_max >= 4 && n_pad_max % 4 == 0, "gs_project_batch: bad n_pad_max=%d", n_pad_max);
  const int nu = probe ? probe->nu : 0;
  const int deg = items[0].x.sh_degree;
  if (deg < 0 || deg > 3 || nu < 0 || nu > 2) {
    gs::set_error("gs_project_batch: unsupported sh_degree=%d nu=%d", deg, nu);
    return GS_ERR_UNSUPPORTED;
  }
  GS_REQUIRE(nu == 0 || out->tangent, "gs_project_batch: probes given but out->tangent is NULL");
  for (int b = 0; b < n_items; ++b) {
    const gs_batch_item& it = items[b];
    GS_REQUIRE(it.x.data && it.cam, "gs_project_batch: item %d has a null buffer", b);
    GS_REQUIRE(it.x.sh_degree == deg, "gs_project_batch: items differ in SH degree");
    GS_REQUIRE(it.x.n >= 0 && it.x.n <= n_pad_max && it.x.n_pad >= it.x.n && it.x.n_pad % 4 == 0,
               "gs_project_batch: item %d has n=%d n_pad=%d for n_pad_max=%d", b, it.x.n, it.x.n_pad, n_pad_max);
    GS_REQUIRE(nu == 0 || it.t >= 1, "gs_project_batch: item %d needs t >= 1 with probes", b);
  }
  const int per_item = (n_pad_max + 127) / 128;
  const gs::BatchArg ba = gs::batch_arg(items, n_items, [&](const gs_batch_item&) { return per_item; });
  gs::ProbeArg pa = gs::probe_arg(probe);
  cudaStream_t st = (cudaStream_t)stream;
  switch (deg) {
    case 0: gs::dispatch_batch<0>(nu, ba, n_pad_max, frame, pa, out, st); break;
    case 1: gs::dispatch_batch<1>(nu, ba, n_pad_max, frame, pa, out, st); break;
    case 2: gs::dispatch_batch<2>(nu, ba, n_pad_max, frame, pa, out, st); break;
    default: gs::dispatch_batch<3>(nu, ba, n_pad_max, frame, pa, out, st); break;
  }
  return gs::check_launch("gs_project_batch");
}
