// gs_tr_update: Algorithm 1 of arXiv 2602.00395 fused into one streaming pass,
// with the per-parameter squared-Hellinger trust-region radius of Sec. 4.2 and
// Appendix B.
//
// A block owns 256 consecutive Gaussians: first the per-Gaussian geometry the
// radii need (alpha, scales, rotation, Sigma_cc, beta_c, DC colour) is turned
// into 14 radii in shared memory, from x_t; then the block streams all 11 + 3K
// rows of its columns with float4 accesses: read x, g_ema, d_ema, grad (and hz
// on curvature steps), write x, g_ema (and d_ema).  The kernel is HBM-bound.
//
// The rotation constant beta_c of Appendix B is evaluated in closed form:
// beta_c = 2 ||S^-1 W_c S||_F^2 - 2 ||W_c||_F^2 = 2 sum_{i<j} W_ij^2 (s_i/s_j - s_j/s_i)^2,
// where W_c = R^T dR/dq_c is skew (its trace term tr(E'') equals -||W_c||_F^2 for
// an orthogonal curve) with axial vector omega_c = 2 vec(conj(q^) * e_c) / |q|.
#include <cmath>

#include "common.cuh"

namespace gs {
namespace {

// max over the unit sphere of |Y_k| (closed forms, one per basis polynomial):
//   |xy|, |yz|, |xz| <= 1/2;  |3z^2 - 1| <= 2;  |x^2 - y^2| <= 1;  |rho^3 sin 3phi| <= 1;
//   |xyz| <= 3^-3/2;  sqrt(1-z^2)|5z^2-1| <= 16/sqrt(135);  |z(5z^2-3)| <= 2;  |z|(1-z^2) <= 2/(3 sqrt 3)
__device__ __forceinline__ float sh_absmax(int k) {
  switch (k) {
    case 0: return kY0;
    case 1: case 2: case 3: return kY1;
    case 4: case 5: case 7: return 0.5f * kY2a;
    case 6: return 2.f * kY2b;
    case 8: return kY2c;
    case 9: case 15: return kY3a;
    case 10: return kY3b * 0.19245008972987526f;       // 3^-3/2
    case 11: case 13: return kY3c * 1.3770607453193149f;  // 16/sqrt(135)
    case 12: return 2.f * kY3d;
    default: return kY3e * 0.38490017945975052f;          // 2/(3 sqrt 3)
  }
}

// One block owns kUpdCols consecutive Gaussians (columns) for all rows.
// Phase 1, one thread per column: the 11 geometric radii and the 3 colour
// radii (before division by max |Y_k|) from x_t into shared memory.  Phase 2:
// the block streams the rows, each thread taking 4 consecutive columns of a row
// (float4), kUpdCols / 4 threads per row and blockDim / (kUpdCols / 4) rows at
// a time.  The radii are read before any column of the block is written, and
// no other block touches these columns, so every radius is that of x_t.
constexpr int kUpdCols = 256;
constexpr int kEtaRows = kRowSH + 3;

__device__ __forceinline__ void radii_of_column(const float* __restrict__ x, int i, int n_pad, const gs_tr_config& cfg,
                                                float eps, float (&eta)[kEtaRows]) {
  auto at = [&](int r) { return (size_t)r * n_pad + i; };
  const float logit = x[at(10)];
  const float alpha = 1.f / (1.f + expf(-logit));
  const float alpha_c = 1.f / (1.f + expf(logit));  // 1 - alpha without cancellation
  float s[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) s[a] = expf(x[at(3 + a)]);
  const float q0 = x[at(6)], q1 = x[at(7)], q2 = x[at(8)], q3 = x[at(9)];
  const float qlen = sqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
  const float X = q0 / qlen, Y = q1 / qlen, Z = q2 / qlen, W = q3 / qlen;
  float R[3][3];
  R[0][0] = 1.f - 2.f * (Y * Y + Z * Z);
  R[0][1] = 2.f * (X * Y - W * Z);
  R[0][2] = 2.f * (X * Z + W * Y);
  R[1][0] = 2.f * (X * Y + W * Z);
  R[1][1] = 1.f - 2.f * (Z * Z + X * X);
  R[1][2] = 2.f * (Y * Z - W * X);
  R[2][0] = 2.f * (X * Z - W * Y);
  R[2][1] = 2.f * (Y * Z + W * X);
  R[2][2] = 1.f - 2.f * (X * X + Y * Y);
  const bool logok = alpha > eps;
  const float L = logok ? log1pf(-eps / alpha) : 0.f;  // ln(1 - eps/alpha)
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float var;
    if (cfg.mean_exact) {
      const float inv = R[c][0] * R[c][0] / (s[0] * s[0]) + R[c][1] * R[c][1] / (s[1] * s[1]) +
                        R[c][2] * R[c][2] / (s[2] * s[2]);
      var = 1.f / inv;
    } else {
      var = R[c][0] * R[c][0] * s[0] * s[0] + R[c][1] * R[c][1] * s[1] * s[1] + R[c][2] * R[c][2] * s[2] * s[2];
    }
    eta[c] = logok ? sqrtf(-8.f * var * L) : INFINITY;
    eta[3 + c] = sqrtf(2.f * eps / alpha);
  }
  {
    // body-frame angular velocity per unit change of q_c (x, y, z, w)
    const float k2 = 2.f / qlen;
    const float om[4][3] = {{W, -Z, Y}, {Z, W, -X}, {-Y, X, W}, {-X, -Y, -Z}};
    const float r01 = s[0] / s[1] - s[1] / s[0];
    const float r02 = s[0] / s[2] - s[2] / s[0];
    const float r12 = s[1] / s[2] - s[2] / s[1];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float w0 = k2 * om[c][0], w1 = k2 * om[c][1], w2 = k2 * om[c][2];
      const float beta = 2.f * (w2 * w2 * r01 * r01 + w1 * w1 * r02 * r02 + w0 * w0 * r12 * r12);
      eta[6 + c] = (logok && beta > 0.f) ? sqrtf(-8.f / beta * L) : INFINITY;
    }
  }
  eta[10] = sqrtf(4.f * alpha * eps) / (alpha * alpha_c);
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    const float Cc = fmaxf(kY0 * x[at(kRowSH + ch)] + 0.5f, cfg.color_floor);
    eta[kRowSH + ch] = sqrtf(4.f * Cc * eps / alpha);
  }
}

// eps_t of the schedule, in double precision, rounded to float
__device__ __forceinline__ float eps_of(const gs_eps_schedule& sc, int64_t t) {
  if (sc.total <= 1) return (float)sc.eps0;
  return (float)(sc.eps0 * pow(sc.eps1 / sc.eps0, (double)(t - 1) / (double)(sc.total - 1)));
}

// HVP: hz is given.  With t_dev the step index is read on the device, eps is
// eps_t of `sched` and d_ema is updated when (t - 1) % l == 0; otherwise eps is
// as passed and d_ema is updated whenever HVP.
// Adam state of the ADAM-TR step (ge holds m, de holds v).
struct AdamArg {
  float b1, b2, eps_adam, inv_bc1, inv_bc2;
  float lr[6];
};

__device__ __forceinline__ int row_group(int r) {
  return r < 3 ? 0 : r < 6 ? 1 : r < 10 ? 2 : r < 11 ? 3 : r < 14 ? 4 : 5;
}

// The columns [c0, c0 + kUpdCols) of one scene (n Gaussians, pitch n_pad):
// phase 1 and phase 2 above.  hvp_now: this step takes d_ema from hz.
template <int DEG, bool HVP, bool ETA, bool ADAM>
__device__ __forceinline__ void tr_update_columns(float* __restrict__ x, float* __restrict__ ge,
                                                  float* __restrict__ de, const float* __restrict__ g,
                                                  const float* __restrict__ hz, float* __restrict__ eta_out, int n,
                                                  int n_pad, const gs_tr_config& cfg, float eps, bool hvp_now,
                                                  const AdamArg& adam, int c0, int32_t* status) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  constexpr int ROWS = kRowSH + 3 * K;
  constexpr int kLanesPerRow = kUpdCols / 4;  // 64
  __shared__ __align__(16) float s_eta[kEtaRows][kUpdCols];
  // phase 1: radii of this block's columns, from x_t
  {
    const int i = c0 + (int)threadIdx.x;
    float eta[kEtaRows];
    if (i < n) {
      radii_of_column(x, i, n_pad, cfg, eps, eta);
    } else {
#pragma unroll
      for (int q = 0; q < kEtaRows; ++q) eta[q] = 0.f;
    }
#pragma unroll
    for (int q = 0; q < kEtaRows; ++q) s_eta[q][threadIdx.x] = eta[q];
  }
  __syncthreads();
  // phase 2: every row of the block's columns, 4 columns per thread
  const int lane4 = (int)threadIdx.x % kLanesPerRow, row0 = (int)threadIdx.x / kLanesPerRow;
  const int rstep = (int)blockDim.x / kLanesPerRow;
  const int ci = c0 + 4 * lane4;  // first of this thread's 4 columns (n_pad % 4 == 0)
  const float a1 = cfg.theta1, b1 = 1.f - cfg.theta1;
  const float a2 = cfg.theta2, b2 = 1.f - cfg.theta2;
  bool bad = false;
  if (ci < n) {
#pragma unroll 4
    for (int r = row0; r < ROWS; r += rstep) {
      int q = r;
      float scale = 1.f;
      if (r >= kRowSH) {
        q = kRowSH + (r - kRowSH) % 3;
        scale = 1.f / sh_absmax((r - kRowSH) / 3);
      }
      const float4 e4 = *reinterpret_cast<const float4*>(&s_eta[q][4 * lane4]);
      const size_t j = (size_t)r * n_pad + ci;
      const float4 x4 = *reinterpret_cast<const float4*>(x + j);
      const float4 ge4 = *reinterpret_cast<const float4*>(ge + j);
      const float4 g4 = *reinterpret_cast<const float4*>(g + j);
      const float4 de4 = *reinterpret_cast<const float4*>(de + j);
      float4 hz4 = make_float4(0.f, 0.f, 0.f, 0.f);
      if (HVP && hvp_now) hz4 = *reinterpret_cast<const float4*>(hz + j);
      const float ev[4] = {e4.x * scale, e4.y * scale, e4.z * scale, e4.w * scale};
      const float xv[4] = {x4.x, x4.y, x4.z, x4.w}, gev[4] = {ge4.x, ge4.y, ge4.z, ge4.w};
      const float gv[4] = {g4.x, g4.y, g4.z, g4.w}, hv[4] = {hz4.x, hz4.y, hz4.z, hz4.w};
      const float dv0[4] = {de4.x, de4.y, de4.z, de4.w};
      float xo[4], go[4], dn[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const bool live = ci + k < n;  // padding columns stay as they are
        float step;
        if constexpr (ADAM) {
          go[k] = live ? adam.b1 * gev[k] + (1.f - adam.b1) * gv[k] : gev[k];
          dn[k] = live ? adam.b2 * dv0[k] + (1.f - adam.b2) * gv[k] * gv[k] : dv0[k];
          step = -adam.lr[row_group(r)] * (go[k] * adam.inv_bc1) / (sqrtf(dn[k] * adam.inv_bc2) + adam.eps_adam);
        } else {
          go[k] = live ? a1 * gev[k] + b1 * gv[k] : gev[k];
          dn[k] = (hvp_now && live) ? a2 * dv0[k] + b2 * hv[k] : dv0[k];
          step = -go[k] / fmaxf(dn[k], cfg.d_floor);
        }
        xo[k] = live ? xv[k] + fminf(fmaxf(step, -ev[k]), ev[k]) : xv[k];
        if (live) bad = bad || !isfinite(xo[k]) || !isfinite(go[k]) || !isfinite(dn[k]);
      }
      *reinterpret_cast<float4*>(x + j) = make_float4(xo[0], xo[1], xo[2], xo[3]);
      *reinterpret_cast<float4*>(ge + j) = make_float4(go[0], go[1], go[2], go[3]);
      if (ADAM || (HVP && hvp_now)) *reinterpret_cast<float4*>(de + j) = make_float4(dn[0], dn[1], dn[2], dn[3]);
      if (ETA) *reinterpret_cast<float4*>(eta_out + j) = make_float4(ev[0], ev[1], ev[2], ev[3]);
    }
  }
  if (bad && status) atomicOr(status, GS_FLAG_NONFINITE);
}

template <int DEG, bool HVP, bool ETA, bool ADAM = false>
__global__ void __launch_bounds__(256) tr_update_kernel(float* __restrict__ x, float* __restrict__ ge,
                                                        float* __restrict__ de, const float* __restrict__ g,
                                                        const float* __restrict__ hz, float* __restrict__ eta_out,
                                                        int n, int n_pad, gs_tr_config cfg, float eps,
                                                        const int64_t* __restrict__ t_dev, gs_eps_schedule sched,
                                                        AdamArg adam, int32_t* status) {
  bool hvp_now = HVP;
  if (t_dev) {
    const int64_t t = *t_dev;
    if (t < 1) {
      if (blockIdx.x == 0 && threadIdx.x == 0 && status) atomicOr(status, GS_FLAG_NONFINITE);
      return;
    }
    eps = eps_of(sched, t);
    hvp_now = HVP && ((t - 1) % cfg.l) == 0;
  }
  tr_update_columns<DEG, HVP, ETA, ADAM>(x, ge, de, g, hz, eta_out, n, n_pad, cfg, eps, hvp_now, adam,
                                         (int)blockIdx.x * kUpdCols, status);
}

// A batch: item b's share of the grid updates its scene with its own eps and
// curvature decision.
template <int DEG>
__global__ void __launch_bounds__(256) tr_update_batch_kernel(BatchArg ba, gs_tr_config cfg, int32_t* status) {
  const int b = batch_item(ba, (int)blockIdx.x);
  const int c0 = ((int)blockIdx.x - ba.first_block[b]) * kUpdCols;
  // the item's x was given as a writable gs_params (BatchArg keeps it as const)
  tr_update_columns<DEG, true, false, false>(const_cast<float*>(ba.P[b]), ba.ge[b], ba.de[b], ba.grad[b], ba.hz[b],
                                             nullptr, ba.n[b], ba.n_pad[b], cfg, ba.eps[b], ba.hvp[b] != 0,
                                             AdamArg{}, c0, status);
}

template <int DEG>
void launch_update(bool hvp, bool eta, gs_params* x, gs_params* ge, gs_params* de, const gs_params* g,
                   const gs_params* hz, gs_params* eta_out, gs_tr_config cfg, float eps, const int64_t* t_dev,
                   gs_eps_schedule sched, int32_t* status, cudaStream_t st) {
  const int blocks = (x->n + kUpdCols - 1) / kUpdCols;
  const float* hp = hz ? hz->data : nullptr;
  float* ep = eta_out ? eta_out->data : nullptr;
#define GS_UPD(H, E)                                                                                         \
  tr_update_kernel<DEG, H, E><<<blocks, 256, 0, st>>>(x->data, ge->data, de->data, g->data, hp, ep, x->n, \
                                                      x->n_pad, cfg, eps, t_dev, sched, AdamArg{}, status)
  if (hvp) {
    if (eta) GS_UPD(true, true); else GS_UPD(true, false);
  } else {
    if (eta) GS_UPD(false, true); else GS_UPD(false, false);
  }
#undef GS_UPD
}

}  // namespace
}  // namespace gs

namespace gs {
namespace {
template <int DEG>
void launch_adam(bool eta, gs_params* x, gs_params* m, gs_params* v, const gs_params* g, gs_params* eta_out,
                 gs_tr_config cfg, float eps, AdamArg adam, int32_t* status, cudaStream_t st) {
  const int blocks = (x->n + kUpdCols - 1) / kUpdCols;
  float* ep = eta_out ? eta_out->data : nullptr;
  const gs_eps_schedule none{0.0, 0.0, 0};
  if (eta)
    tr_update_kernel<DEG, false, true, true><<<blocks, 256, 0, st>>>(x->data, m->data, v->data, g->data, nullptr, ep,
                                                                    x->n, x->n_pad, cfg, eps, nullptr, none, adam,
                                                                    status);
  else
    tr_update_kernel<DEG, false, false, true><<<blocks, 256, 0, st>>>(x->data, m->data, v->data, g->data, nullptr,
                                                                     nullptr, x->n, x->n_pad, cfg, eps, nullptr, none,
                                                                     adam, status);
}

__global__ void step_advance_kernel(int64_t* t) { *t += 1; }

gs_status run_update(const char* name, gs_params* x, gs_params* g_ema, gs_params* d_ema, const gs_params* grad,
                     const gs_params* hz, const gs_tr_config* cfg, bool hvp, float eps, const int64_t* t_dev,
                     gs_eps_schedule sched, gs_params* eta_out, int32_t* status, void* stream) {
  GS_REQUIRE(x && g_ema && d_ema && grad && cfg, "%s: null argument", name);
  GS_REQUIRE(x->data && g_ema->data && d_ema->data && grad->data, "%s: null device buffer", name);
  GS_REQUIRE(cfg->l >= 1, "%s: need l >= 1", name);
  auto same = [&](const gs_params* p) {
    return !p || (p->n == x->n && p->n_pad == x->n_pad && p->sh_degree == x->sh_degree);
  };
  GS_REQUIRE(same(g_ema) && same(d_ema) && same(grad) && same(hz) && same(eta_out),
             "%s: parameter buffers differ in layout", name);
  GS_REQUIRE(x->n_pad % 4 == 0, "%s: n_pad must be a multiple of 4", name);
  if (x->sh_degree < 0 || x->sh_degree > 3) {
    set_error("%s: unsupported sh_degree=%d", name, x->sh_degree);
    return GS_ERR_UNSUPPORTED;
  }
  if (x->n == 0) return GS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const bool eta = eta_out && eta_out->data;
  switch (x->sh_degree) {
    case 0: launch_update<0>(hvp, eta, x, g_ema, d_ema, grad, hz, eta_out, *cfg, eps, t_dev, sched, status, st); break;
    case 1: launch_update<1>(hvp, eta, x, g_ema, d_ema, grad, hz, eta_out, *cfg, eps, t_dev, sched, status, st); break;
    case 2: launch_update<2>(hvp, eta, x, g_ema, d_ema, grad, hz, eta_out, *cfg, eps, t_dev, sched, status, st); break;
    default: launch_update<3>(hvp, eta, x, g_ema, d_ema, grad, hz, eta_out, *cfg, eps, t_dev, sched, status, st); break;
  }
  return check_launch(name);
}
}  // namespace
}  // namespace gs

extern "C" gs_status gs_tr_update(gs_params* x, gs_params* g_ema, gs_params* d_ema, const gs_params* grad,
                                  const gs_params* hz, const gs_tr_config* cfg, int64_t t, float eps,
                                  gs_params* eta_out, int32_t* status, void* stream) {
  using namespace gs;
  GS_REQUIRE(cfg, "gs_tr_update: null argument");
  GS_REQUIRE(t >= 1 && cfg->l >= 1, "gs_tr_update: need t >= 1 and l >= 1");
  GS_REQUIRE(eps > 0.f, "gs_tr_update: eps must be positive");
  const bool hvp = ((t - 1) % cfg->l) == 0 && hz && hz->data;
  const gs_eps_schedule none{0.0, 0.0, 0};
  return run_update("gs_tr_update", x, g_ema, d_ema, grad, hz, cfg, hvp, eps, nullptr, none, eta_out, status,
                    stream);
}

extern "C" gs_status gs_tr_update_dev(gs_params* x, gs_params* g_ema, gs_params* d_ema, const gs_params* grad,
                                      const gs_params* hz, const gs_tr_config* cfg, const int64_t* t_device,
                                      const gs_eps_schedule* schedule, gs_params* eta_out, int32_t* status,
                                      void* stream) {
  using namespace gs;
  GS_REQUIRE(cfg && t_device && schedule, "gs_tr_update_dev: null argument");
  GS_REQUIRE(schedule->eps0 > 0.0 && schedule->eps1 > 0.0, "gs_tr_update_dev: eps0 and eps1 must be positive");
  const bool hvp = hz && hz->data;
  return run_update("gs_tr_update_dev", x, g_ema, d_ema, grad, hz, cfg, hvp, 0.f, t_device, *schedule, eta_out,
                    status, stream);
}

extern "C" gs_status gs_step_advance(int64_t* t_device, void* stream) {
  using namespace gs;
  GS_REQUIRE(t_device, "gs_step_advance: null argument");
  step_advance_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(t_device);
  return check_launch("gs_step_advance");
}

extern "C" gs_status gs_adam_tr_update(gs_params* x, gs_params* m, gs_params* v, const gs_params* grad,
                                       const gs_tr_config* cfg, const gs_adam_config* adam, int64_t t, float eps,
                                       gs_params* eta_out, int32_t* status, void* stream) {
  using namespace gs;
  GS_REQUIRE(x && m && v && grad && cfg && adam, "gs_adam_tr_update: null argument");
  GS_REQUIRE(x->data && m->data && v->data && grad->data, "gs_adam_tr_update: null device buffer");
  GS_REQUIRE(t >= 1, "gs_adam_tr_update: need t >= 1");
  GS_REQUIRE(eps > 0.f, "gs_adam_tr_update: eps must be positive");
  GS_REQUIRE(adam->beta1 >= 0.f && adam->beta1 < 1.f && adam->beta2 >= 0.f && adam->beta2 < 1.f,
             "gs_adam_tr_update: betas must be in [0, 1)");
  auto same = [&](const gs_params* p) {
    return !p || (p->n == x->n && p->n_pad == x->n_pad && p->sh_degree == x->sh_degree);
  };
  GS_REQUIRE(same(m) && same(v) && same(grad) && same(eta_out), "gs_adam_tr_update: buffers differ in layout");
  GS_REQUIRE(x->n_pad % 4 == 0, "gs_adam_tr_update: n_pad must be a multiple of 4");
  if (x->sh_degree < 0 || x->sh_degree > 3) {
    set_error("gs_adam_tr_update: unsupported sh_degree=%d", x->sh_degree);
    return GS_ERR_UNSUPPORTED;
  }
  if (x->n == 0) return GS_OK;
  AdamArg a;
  a.b1 = adam->beta1;
  a.b2 = adam->beta2;
  a.eps_adam = adam->eps_adam;
  // bias corrections of step t, in double precision on the host
  a.inv_bc1 = (float)(1.0 / (1.0 - std::pow((double)adam->beta1, (double)t)));
  a.inv_bc2 = (float)(1.0 / (1.0 - std::pow((double)adam->beta2, (double)t)));
  for (int q = 0; q < 6; ++q) a.lr[q] = adam->lr[q];
  const bool eta = eta_out && eta_out->data;
  cudaStream_t st = (cudaStream_t)stream;
  switch (x->sh_degree) {
    case 0: launch_adam<0>(eta, x, m, v, grad, eta_out, *cfg, eps, a, status, st); break;
    case 1: launch_adam<1>(eta, x, m, v, grad, eta_out, *cfg, eps, a, status, st); break;
    case 2: launch_adam<2>(eta, x, m, v, grad, eta_out, *cfg, eps, a, status, st); break;
    default: launch_adam<3>(eta, x, m, v, grad, eta_out, *cfg, eps, a, status, st); break;
  }
  return check_launch("gs_adam_tr_update");
}

extern "C" gs_status gs_tr_update_batch(const gs_batch_item* items, int32_t n_items, const gs_tr_config* cfg,
                                        int32_t* status, void* stream) {
  using namespace gs;
  const char* name = "gs_tr_update_batch";
  GS_REQUIRE(items && cfg, "%s: null argument", name);
  GS_REQUIRE(n_items >= 1 && n_items <= GS_BATCH_MAX, "%s: n_items=%d outside [1, %d]", name, n_items, GS_BATCH_MAX);
  GS_REQUIRE(cfg->l >= 1, "%s: need l >= 1", name);
  const int deg = items[0].x.sh_degree;
  if (deg < 0 || deg > 3) {
    set_error("%s: unsupported sh_degree=%d", name, deg);
    return GS_ERR_UNSUPPORTED;
  }
  for (int b = 0; b < n_items; ++b) {
    const gs_batch_item& it = items[b];
    auto same = [&](const gs_params& p) { return p.n == it.x.n && p.n_pad == it.x.n_pad && p.sh_degree == deg; };
    GS_REQUIRE(it.x.data && it.g_ema.data && it.d_ema.data && it.grad.data, "%s: item %d has a null buffer", name,
               b);
    GS_REQUIRE(same(it.x) && same(it.g_ema) && same(it.d_ema) && same(it.grad), "%s: item %d: buffers differ in layout",
               name, b);
    GS_REQUIRE(!it.hvp || (it.hz.data && same(it.hz)), "%s: item %d takes curvature but has no hz", name, b);
    GS_REQUIRE(it.x.n_pad % 4 == 0 && it.t >= 1 && it.eps > 0.f, "%s: item %d: bad n_pad, t or eps", name, b);
  }
  const BatchArg ba = batch_arg(items, n_items, [](const gs_batch_item& it) {
    return (it.x.n + kUpdCols - 1) / kUpdCols;
  });
  const int blocks = ba.first_block[n_items];
  if (blocks == 0) return GS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  switch (deg) {
    case 0: tr_update_batch_kernel<0><<<blocks, 256, 0, st>>>(ba, *cfg, status); break;
    case 1: tr_update_batch_kernel<1><<<blocks, 256, 0, st>>>(ba, *cfg, status); break;
    case 2: tr_update_batch_kernel<2><<<blocks, 256, 0, st>>>(ba, *cfg, status); break;
    default: tr_update_batch_kernel<3><<<blocks, 256, 0, st>>>(ba, *cfg, status); break;
  }
  return check_launch(name);
}
