// Rasteriser forward and reverse passes of arXiv 2602.00395:
//
//   gs_raster_fwd  front-to-back alpha blending per pixel (Sec. 3.1), with the
//                  forward-mode tangents J z_k of the Hutchinson probes fused in
//                  (Sec. 4.1; the paper's forward-mode AD of the rasteriser, Sec. 5)
//   gs_raster_bwd  reverse pass for the gradient g = (1/m) J^T F (Sec. 4.1) and,
//                  in the same sweep, the Gauss-Newton products J^T diag(w) J z_k
//   gs_hvp_diag    the Gauss-Newton products alone
//
// One CTA renders one tile of one view with two pixels per thread; each warp
// owns an 8 x 8 pixel block.  The tile's splat records are staged through
// shared memory in batches (one record per pixel of the tile), each record moved
// by a 48-byte TMA bulk copy (cp.async.bulk, no multicast) completing on an
// mbarrier, double-buffered so that the next batch lands while the current one
// is blended.  Per batch every splat gets a mask of the warp blocks its
// alpha >= 1/255 footprint can reach, and each warp walks only its own visible
// splats (one ballot per 32).  In the reverse pass the warps release the two
// buffers one by one instead of meeting at block barriers, and the last warp
// out refills a buffer.  The reverse pass walks the list back to front,
// recovers T_i = T_{i+1} / (1 - a_i) from the final transmittance (nothing per
// pair is stored), sums each splat's 9 x streams partial derivatives over the
// warp's 64 pixels with a reduction that ends in quads, and adds them with float4
// atomics.  The projection's reverse pass (2-D cotangents -> 11 + 3K parameter
// rows) runs one thread per Gaussian and sums over the views.
#include "common.cuh"

namespace gs {
namespace {

struct alignas(16) Rec {
  float4 a;  // mx, my, A, B
  float4 b;  // C, opacity, r, g
  float4 c;  // b, depth, radius bits, unused
};
static_assert(sizeof(Rec) == 48, "record size");

// Power and alpha of a splat at a pixel with a fixed rounding sequence, so that
// the forward and reverse kernels take identical decisions.
__device__ __forceinline__ float splat_power(const Rec& r, float dx, float dy) {
  const float q = __fmaf_rn(r.b.x, __fmul_rn(dy, dy), __fmul_rn(r.a.z, __fmul_rn(dx, dx)));
  return __fmaf_rn(-0.5f, q, -__fmul_rn(r.a.w, __fmul_rn(dx, dy)));
}

// 1: the blends also test a splat's footprint ellipse itself, not only its
// bounding box, against each 8 x 8 pixel block (0: the box alone).
#ifndef GS_EXACT_BLOCK_TEST
#define GS_EXACT_BLOCK_TEST 1
#endif

// False only if no pixel centre of the 8 x 8 block with first centre (x0, y0)
// can reach alpha >= 1/255: the minimum over the rectangle [x0, x0 + 7] x
// [y0, y0 + 7] of q(u) = A ux^2 + 2 B ux uy + C uy^2, u = p - mean (-2 x the
// power), is above 2 ln(255 o) by more than a slack that covers the FP32
// rounding of both this test and the blends' own evaluation (1e-4 of the
// terms' largest magnitude on the rectangle, 1e-3 relative and absolute, each
// hundreds of times their error bounds).  With the origin outside the rectangle
// the convex q takes its minimum on an edge, where it is a parabola in one
// coordinate.  A conic that is not positive definite is never rejected.
__device__ __forceinline__ bool footprint_meets_block(const Rec& r, float x0, float y0) {
  const float A = r.a.z, B = r.a.w, C = r.b.x;
  if (!(A > 0.f && C > 0.f && A * C > B * B)) return true;
  const float thr = 2.f * __logf(255.f * r.b.y);
  const float xl = x0 - r.a.x, xh = xl + 7.f, yl = y0 - r.a.y, yh = yl + 7.f;
  const float X = fmaxf(fabsf(xl), fabsf(xh)), Y = fmaxf(fabsf(yl), fabsf(yh));
  const float slack = 1e-4f * (A * X * X + 2.f * fabsf(B) * X * Y + C * Y * Y) + 1e-3f * fabsf(thr) + 1e-3f;
  if (xl <= 0.f && xh >= 0.f && yl <= 0.f && yh >= 0.f) return thr + slack >= 0.f;
  const float bc = B / C, ba = B / A;
  auto on_x_edge = [&](float ux) {  // q on ux = const, minimised over uy in [yl, yh]
    const float uy = fminf(fmaxf(-bc * ux, yl), yh);
    return A * ux * ux + 2.f * B * ux * uy + C * uy * uy;
  };
  auto on_y_edge = [&](float uy) {
    const float ux = fminf(fmaxf(-ba * uy, xl), xh);
    return A * ux * ux + 2.f * B * ux * uy + C * uy * uy;
  };
  const float qmin = fminf(fminf(on_x_edge(xl), on_x_edge(xh)), fminf(on_y_edge(yl), on_y_edge(yh)));
  return qmin <= thr + slack;
}

// Stage batch b of a tile list (records [b * batch, b * batch + batch)) into
// buffer (b & 1): one bulk copy per splat, of its record alone (NT = 0, from
// rec) or of its record and NT probe tangent records (from tan, where they are
// adjacent; staged as [batch][1 + NT]), issued by the block's threads in turn,
// all completing on the buffer's mbarrier.
template <int NT>
__device__ __forceinline__ void stage_batch(int b, int batch, uint32_t start, int n, int view, int n_pad,
                                            const uint32_t* __restrict__ vals, const float4* __restrict__ rec,
                                            const float4* __restrict__ tan, Rec* buf, uint32_t* s_idx,
                                            uint64_t* bars) {
  const int bi = b & 1;
  const int cnt = min(batch, n - b * batch);
  if (threadIdx.x == 0) mbar_arrive_expect_tx(&bars[bi], (uint32_t)(cnt * (int)sizeof(Rec) * (1 + NT)));
  fence_proxy_async();
  for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
    const uint32_t gi = vals[start + (uint32_t)(b * batch + q)];
    if (s_idx) s_idx[bi * batch + q] = gi;
    if (NT > 0)  // the record and its NT probe tangent records, adjacent in tan: one copy
      bulk_g2s(&buf[((size_t)bi * batch + q) * (1 + NT)], tan + 3 * ((size_t)view * n_pad + gi) * (1 + NT),
               (1 + NT) * sizeof(Rec), &bars[bi]);
    else
      bulk_g2s(&buf[bi * batch + q], rec + 3 * ((size_t)view * n_pad + gi), sizeof(Rec), &bars[bi]);
  }
}

// ------------------------------------------------------------ pixel blocks
// A tile has tile_w x tile_h pixels and half as many threads: each warp covers
// an 8 x 8 pixel block, warp w the block (w % (tile_w/8), w / (tile_w/8)), and
// its lane renders pixels (lx, ly) and (lx, ly + 4) of it.  Compact blocks meet
// few splats; two pixels per thread halve the per-splat warp overheads.
constexpr int kPixPerThread = 2;
// Records staged per batch, per thread (when the frame leaves the batch at 0).
#ifndef GS_BATCH_PER_THREAD
#define GS_BATCH_PER_THREAD 1
#endif
constexpr int kBatchPerThread = GS_BATCH_PER_THREAD;
// The forward pass stages nthr / kFwdBatchDiv records per batch (its tangent
// records triple the shared memory of a batch).
#ifndef GS_FWD_BATCH_DIV
#define GS_FWD_BATCH_DIV 1
#endif
constexpr int kFwdBatchDiv = GS_FWD_BATCH_DIV;
__host__ __device__ __forceinline__ int fwd_batch(const gs_frame& fr, int nthr) {
  return fr.batch ? fr.batch : kBatchPerThread * nthr / kFwdBatchDiv;
}
__host__ __device__ __forceinline__ int bwd_batch(const gs_frame& fr, int nthr) {
  return fr.batch ? fr.batch : kBatchPerThread * nthr;
}
// Minimum resident CTAs per SM requested for the forward kernel (0: none), for
// blocks of 128 threads; blocks of NT threads (tiles of 2 NT pixels) request
// the same threads per SM.  Six (80 registers, a few bytes spilled) measured
// 9 % faster than the five that 93 unbounded registers allow; seven spilled
// more and gained less.
#ifndef GS_FWD_MIN_BLOCKS
#define GS_FWD_MIN_BLOCKS 6
#endif
#if GS_FWD_MIN_BLOCKS > 0
#define GS_FWD_BOUNDS(NT) __launch_bounds__(NT, (GS_FWD_MIN_BLOCKS * 128) / (NT))
#else
#define GS_FWD_BOUNDS(NT) __launch_bounds__(NT)
#endif
// Threads per block the blends are built for: tiles of up to 256 pixels run
// as blocks of at most 128 threads, tiles of 512 pixels as blocks of 256.
__host__ __device__ constexpr int blend_threads(int nthr) { return nthr <= 128 ? 128 : 256; }

__device__ __forceinline__ void pixel_of(int tid, int tile_w, int& lx, int& ly) {
  const int warp = tid >> 5, lane = tid & 31, bxn = tile_w >> 3;
  lx = (warp % bxn) * 8 + (lane & 7);
  ly = (warp / bxn) * 8 + (lane >> 3);
}

// Bit w is set if the splat can reach alpha >= 1/255 at some pixel centre of
// warp block w.  The record's last word holds the half-extents of the bounding
// box of that footprint, widened and rounded up by the projection
// (footprint_extents); a block inside the box is then tested against the
// ellipse (footprint_meets_block).  Both tests are conservative, so a cleared
// bit skips only pairs that every pixel of the block skips anyway: results are
// unchanged.
__device__ __forceinline__ uint32_t warp_block_mask(const Rec& r, float tile_x0, float tile_y0, int tile_w,
                                                    int nwarps) {
  const uint32_t e = __float_as_uint(r.c.w);
  const float hx = __half2float(__ushort_as_half((unsigned short)(e & 0xffffu)));
  const float hy = __half2float(__ushort_as_half((unsigned short)(e >> 16)));
  const int bxn = tile_w >> 3;
  uint32_t m = 0;
  for (int w = 0; w < nwarps; ++w) {
    const float x0 = tile_x0 + (float)((w % bxn) * 8) + 0.5f, x1 = x0 + 7.f;
    const float y0 = tile_y0 + (float)((w / bxn) * 8) + 0.5f, y1 = y0 + 7.f;
    if (r.a.x + hx >= x0 && r.a.x - hx <= x1 && r.a.y + hy >= y0 && r.a.y - hy <= y1 &&
        (!GS_EXACT_BLOCK_TEST || footprint_meets_block(r, x0, y0)))
      m |= 1u << w;
  }
  return m;
}

// ------------------------------------------------------------------ forward
// Blend state of one pixel: colour, transmittance, the probe tangents of both,
// and the list position after the last blended splat.
template <int NU>
struct FwdPixel {
  float C[3], T;
  float Cd[NU > 0 ? NU : 1][3], Td[NU > 0 ? NU : 1];
  float pxc, pyc;
  uint32_t last;
  bool done;
};

// The splat at one pixel: offsets, Gaussian, alpha, and whether it is blended
// there (a done pixel blends nothing).
template <int NU>
__device__ __forceinline__ bool fwd_eval(const FwdPixel<NU>& p, const Rec& r, float& dx, float& dy, float& G,
                                         float& oG, float& alpha) {
  dx = __fsub_rn(r.a.x, p.pxc);
  dy = __fsub_rn(r.a.y, p.pyc);
  const float power = splat_power(r, dx, dy);
  G = __expf(power);
  oG = __fmul_rn(r.b.y, G);
  alpha = fminf(kAlphaMax, oG);
  return !p.done && power <= 0.f && alpha >= kAlphaMin;
}

// The splat's front-to-back update of one pixel, with the decisions as
// selects: a pixel that does not blend the splat (on false, or the splat would
// take T below kTMin, which ends the pixel instead) adds exact zeros and keeps
// T, its tangents and its last position.  `t0` points at the splat's first
// rewritten tangent record; the records of further probes follow at stride
// `tstride`.  With the power's tangent pd, a blended pixel gets
// C += c a T, C' += c' a T + c (a' T + a T'), T' <- T' (1 - a) - T a', T <- T (1 - a),
// a' = o' G + a pd (0 for a capped alpha).
template <int NU>
__device__ __forceinline__ void fwd_apply(FwdPixel<NU>& p, const Rec& r, const Rec* t0, int tstride, uint32_t pos,
                                          bool on, float dx, float dy, float G, float oG, float alpha) {
  const float Tn = p.T * (1.f - alpha);
  const bool term = on && Tn < kTMin;
  const bool bl = on && !term;
  p.done = p.done || term;
  const float a = bl ? alpha : 0.f;
  const float w = a * p.T;
  if constexpr (NU > 0) {
    const bool live = bl && !(oG > kAlphaMax);  // a capped alpha has no tangent
#pragma unroll
    for (int k = 0; k < NU; ++k) {
      const Rec t = t0[k * tstride];
      const float pd = dx * (t.a.x * dx + t.a.y * dy + t.a.w) + dy * (t.a.z * dy + t.b.x);
      const float ad = live ? (t.b.y * G + alpha * pd) : 0.f;
      const float sk = ad * p.T + a * p.Td[k];
      p.Cd[k][0] += t.b.z * w + r.b.z * sk;
      p.Cd[k][1] += t.b.w * w + r.b.w * sk;
      p.Cd[k][2] += t.c.x * w + r.c.x * sk;
      p.Td[k] = p.Td[k] * (1.f - a) - p.T * ad;
    }
  }
  p.C[0] += r.b.z * w;
  p.C[1] += r.b.w * w;
  p.C[2] += r.c.x * w;
  p.T = bl ? Tn : p.T;
  p.last = bl ? pos + 1 : p.last;
}

// 1: when a batch holds at most one record per thread, each thread reads the
// Gaussian index of its record in the batch after next one iteration ahead, so
// that staging a batch does not wait on that read.
#ifndef GS_FWD_PREFETCH_VALS
#define GS_FWD_PREFETCH_VALS 1
#endif

// stage_batch for a batch of at most blockDim.x records, the calling thread's
// record (threadIdx.x) being splat gi.
template <int NT>
__device__ __forceinline__ void stage_batch_one(int b, int batch, int n, int view, int n_pad, uint32_t gi,
                                                const float4* __restrict__ rec, const float4* __restrict__ tan,
                                                Rec* buf, uint64_t* bars) {
  const int bi = b & 1;
  const int cnt = min(batch, n - b * batch);
  if (threadIdx.x == 0) mbar_arrive_expect_tx(&bars[bi], (uint32_t)(cnt * (int)sizeof(Rec) * (1 + NT)));
  fence_proxy_async();
  const int q = threadIdx.x;
  if (q < cnt) {
    if (NT > 0)  // the record and its NT probe tangent records, adjacent in tan: one copy
      bulk_g2s(&buf[((size_t)bi * batch + q) * (1 + NT)], tan + 3 * ((size_t)view * n_pad + gi) * (1 + NT),
               (1 + NT) * sizeof(Rec), &bars[bi]);
    else
      bulk_g2s(&buf[bi * batch + q], rec + 3 * ((size_t)view * n_pad + gi), sizeof(Rec), &bars[bi]);
  }
}

// CB: the frame sets its own batch (else one record per thread, known to the
// compiler as the block size).
template <int NU, bool CB, int NT>
__global__ void GS_FWD_BOUNDS(NT) raster_fwd_kernel(const float4* __restrict__ rec, const float4* __restrict__ tan,
                                                         const uint32_t* __restrict__ vals,
                                                         const uint32_t* __restrict__ ranges,
                                                         const uint32_t* __restrict__ order, int n_pad, gs_frame fr,
                                                         int Tx, int T, float* __restrict__ image,
                                                         float* __restrict__ final_T, uint32_t* __restrict__ n_contrib,
                                                         float* __restrict__ image_tan, uint8_t* __restrict__ masks,
                                                         int32_t* status) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int nthr = blockDim.x, nwarps = nthr >> 5, batch = CB ? fr.batch : kBatchPerThread * nthr / kFwdBatchDiv;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  Rec* buf = reinterpret_cast<Rec*>(smem + 16);
  uint32_t* s_mask = reinterpret_cast<uint32_t*>(buf + 2 * (1 + NU) * batch);  // after both buffers
  const int tid = threadIdx.x, lane = tid & 31;
  const uint32_t wbit = 1u << (tid >> 5);
  // the tile of this block: the heaviest tiles first when an order is given
  const int blk = order ? (int)min(__ldg(order + blockIdx.x), gridDim.x - 1) : (int)blockIdx.x;
  const int view = blk / T, tile = blk - view * T;
  const int ty = tile / Tx, tx = tile - ty * Tx;
  int lx, ly;
  pixel_of(tid, fr.tile_w, lx, ly);
  const float tile_x0 = (float)(tx * fr.tile_w), tile_y0 = (float)(ty * fr.tile_h);
  const size_t tslot = 2 * ((size_t)view * T + tile);
  const uint32_t start = ranges[tslot], end = ranges[tslot + 1];
  const int n = (int)(end - start);
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  FwdPixel<NU> pix[kPixPerThread];
  int px[kPixPerThread], py[kPixPerThread];
#pragma unroll
  for (int q = 0; q < kPixPerThread; ++q) {
    px[q] = tx * fr.tile_w + lx;
    py[q] = ty * fr.tile_h + ly + 4 * q;
    FwdPixel<NU>& p = pix[q];
    p.C[0] = p.C[1] = p.C[2] = 0.f;
    p.T = 1.f;
#pragma unroll
    for (int k = 0; k < NU; ++k) p.Cd[k][0] = p.Cd[k][1] = p.Cd[k][2] = p.Td[k] = 0.f;
    p.pxc = (float)px[q] + 0.5f;
    p.pyc = (float)py[q] + 0.5f;
    p.last = 0;
    p.done = !(px[q] < fr.width && py[q] < fr.height);
  }
  __syncthreads();

  const int nb = (n + batch - 1) / batch;
  int issued = 0;  // batches staged so far (block-uniform)
  // with at most one record per thread and batch, the index of this thread's
  // record in batch bb (0 past the list), read one batch ahead of its staging
  const bool one = GS_FWD_PREFETCH_VALS && batch <= nthr;
  auto index_of = [&](int bb) -> uint32_t {
    const int q = bb * batch + tid;
    return (bb < nb && tid < batch && q < n) ? __ldg(vals + start + (uint32_t)q) : 0u;
  };
  uint32_t gi_next = 0;
  if (nb > 0) {
    if (one) {
      stage_batch_one<NU>(0, batch, n, view, n_pad, index_of(0), rec, tan, buf, bars);
      gi_next = index_of(1);
    } else {
      stage_batch<NU>(0, batch, start, n, view, n_pad, vals, rec, tan, buf, nullptr, bars);
    }
    issued = 1;
  }
  for (int b = 0; b < nb; ++b) {
    if (b + 1 < nb) {
      if (one) {
        stage_batch_one<NU>(b + 1, batch, n, view, n_pad, gi_next, rec, tan, buf, bars);
        gi_next = index_of(b + 2);
      } else {
        stage_batch<NU>(b + 1, batch, start, n, view, n_pad, vals, rec, tan, buf, nullptr, bars);
      }
      issued = b + 2;
    }
    const int bi = b & 1;
    const bool ok = mbar_wait_bounded(&bars[bi], (uint32_t)((b >> 1) & 1), status);
    const int cnt = min(batch, n - b * batch);
    // record q of the batch; its probe tangent records follow it (NU > 0)
    auto recp = [&](int q) -> Rec* {
      return NU > 0 ? &buf[((size_t)bi * batch + q) * (1 + NU)] : &buf[bi * batch + q];
    };
    // per splat: which warps it can reach, and the probe tangents of its power
    // rewritten as the quadratic form pd = dx (a dx + b dy + d) + dy (c dy + e)
    for (int q = tid; q < cnt; q += nthr) {
      const Rec r = *recp(q);
      s_mask[q] = ok ? warp_block_mask(r, tile_x0, tile_y0, fr.tile_w, nwarps) : 0u;
      if (masks) masks[start + (uint32_t)(b * batch + q)] = (uint8_t)s_mask[q];  // for the reverse passes
#pragma unroll
      for (int k = 0; k < NU; ++k) {
        Rec* tp = recp(q) + 1 + k;
        const float4 ta = tp->a;  // dmx, dmy, dA, dB
        const float dC = tp->b.x;
        tp->a = make_float4(-0.5f * ta.z, -ta.w, -0.5f * dC, -(r.a.z * ta.x + r.a.w * ta.y));
        tp->b.x = -(r.b.x * ta.y + r.a.w * ta.x);
      }
    }
    __syncthreads();
    if (!ok) {
#pragma unroll
      for (int q = 0; q < kPixPerThread; ++q) pix[q].done = true;
    }
    // The warp walks only the splats its block can see: one ballot per 32
    // splats, then the set bits in list order.
    for (int j0 = 0; j0 < cnt; j0 += 32) {
      if (__all_sync(0xffffffffu, pix[0].done && pix[1].done)) break;
      uint32_t bits = __ballot_sync(0xffffffffu, j0 + lane < cnt && (s_mask[j0 + lane] & wbit));
      while (bits) {
        const int j = j0 + __ffs(bits) - 1;
        bits &= bits - 1;
        const Rec r = *recp(j);
        const Rec* t0 = recp(j) + 1;
        const uint32_t pos = (uint32_t)(b * batch + j);
        float dx[kPixPerThread], dy[kPixPerThread], G[kPixPerThread], oG[kPixPerThread], al[kPixPerThread];
        bool on[kPixPerThread];
#pragma unroll
        for (int q = 0; q < kPixPerThread; ++q) on[q] = fwd_eval<NU>(pix[q], r, dx[q], dy[q], G[q], oG[q], al[q]);
        // a pixel row (the lanes' first or second pixels) that no lane blends
        // the splat at is skipped as a whole; the splat's probe tangent records
        // are read once for both rows
        bool rows[kPixPerThread];
        bool anyrow = false;
#pragma unroll
        for (int q = 0; q < kPixPerThread; ++q) {
          rows[q] = __any_sync(0xffffffffu, on[q]);
          anyrow = anyrow || rows[q];
        }
        if (!anyrow) continue;
        Rec tk[NU > 0 ? NU : 1];
#pragma unroll
        for (int k = 0; k < NU; ++k) tk[k] = t0[k];
#pragma unroll
        for (int q = 0; q < kPixPerThread; ++q)
          if (rows[q]) fwd_apply<NU>(pix[q], r, tk, 1, pos, on[q], dx[q], dy[q], G[q], oG[q], al[q]);
      }
    }
    if (__syncthreads_count(pix[0].done && pix[1].done) == nthr) break;
  }
  // Drain: a buffer is refilled only after a barrier that follows every
  // thread's wait on its previous fill, and only when some wait saw that fill
  // land, so each buffer has at most one fill in flight, its last.  Thread 0
  // waits (bounded) for the last fill of both buffers, so that no bulk copy is
  // still writing into this block's shared memory when it exits: the batch
  // staged ahead of an early finish, or a fill whose waits ran out.
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int last = issued - 1 - (((issued - 1) ^ s) & 1);  // largest batch < issued in buffer s
      if (last >= 0) mbar_wait_bounded(&bars[s], (uint32_t)((last >> 1) & 1), status);
    }
  }
  const size_t HW = (size_t)fr.width * fr.height;
#pragma unroll
  for (int q = 0; q < kPixPerThread; ++q) {
    if (!(px[q] < fr.width && py[q] < fr.height)) continue;
    const FwdPixel<NU>& p = pix[q];
    const size_t at = (size_t)py[q] * fr.width + px[q];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) image[((size_t)view * 3 + ch) * HW + at] = p.C[ch];
    final_T[(size_t)view * HW + at] = p.T;
    n_contrib[(size_t)view * HW + at] = p.last;
#pragma unroll
    for (int k = 0; k < NU; ++k)
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) image_tan[(((size_t)k * fr.n_views + view) * 3 + ch) * HW + at] = p.Cd[k][ch];
  }
}

// ------------------------------------------------------------------ reverse
// The reverse pass stages its batches in a ring of kBwdStages buffers that the
// warps release one by one, instead of block barriers per batch: a warp moves
// on to the next batch as soon as it has landed and tests only its own block's
// visibility, so a warp with little work in a batch does not wait for the
// others.  The last warp to release a buffer refills it with the batch
// kBwdStages further on.  At 7 CTAs per SM three stages measured fastest (at
// 8 CTAs per SM two did: deeper rings took shared memory from L1 or from
// resident CTAs).
#ifndef GS_BWD_STAGES
#define GS_BWD_STAGES 3
#endif
constexpr int kBwdStages = GS_BWD_STAGES;
// ring header: one mbarrier and one release counter per stage, 16-byte aligned
constexpr size_t kBwdRingHdr = (kBwdStages * (sizeof(uint64_t) + sizeof(uint32_t)) + 15) / 16 * 16;
__host__ __device__ constexpr size_t bwd_smem_bytes(int batch) {
  return kBwdRingHdr + (size_t)kBwdStages * batch * (sizeof(Rec) + sizeof(uint32_t)) +
         ((size_t)kBwdStages * batch + 15) / 16 * 16;  // and the staged block masks, one byte per record
}

// The calling warp fills ring stage s with batch b of the list (use u of the
// ring): its lanes store the Gaussian indices (and, given the forward pass's
// block masks, each record's mask byte) and issue one bulk copy per record,
// then lane 0 records u as the stage's last fill and arms the stage's barrier
// with the byte count.  The copies may complete before that arrival (the
// phase cannot complete while the arrival is pending), and the arrival releases
// the index stores to the warps that wait on the phase.
__device__ __forceinline__ void stage_batch_warp(int s, int u, int b, int batch, uint32_t start, int n, int view,
                                                 int n_pad, const uint32_t* __restrict__ vals,
                                                 const float4* __restrict__ rec, const uint8_t* __restrict__ masks,
                                                 Rec* buf, uint32_t* s_idx, uint8_t* s_bits, uint64_t* full,
                                                 int* fill_use) {
  const int lane = threadIdx.x & 31;
  const int cnt = min(batch, n - b * batch);
  __syncwarp();
  fence_proxy_async();  // the ring slot's earlier reads come before the copies' writes
  for (int q = lane; q < cnt; q += 32) {
    const uint32_t gi = __ldg(vals + start + (uint32_t)(b * batch + q));
    s_idx[s * batch + q] = gi;
    if (masks) s_bits[s * batch + q] = __ldg(masks + start + (uint32_t)(b * batch + q));
    bulk_g2s(&buf[s * batch + q], rec + 3 * ((size_t)view * n_pad + gi), sizeof(Rec), &full[s]);
  }
  __syncwarp();
  if (lane == 0) {
    fill_use[s] = u;
    mbar_arrive_expect_tx(&full[s], (uint32_t)(cnt * (int)sizeof(Rec)));
  }
}

// True if the splat can reach alpha >= 1/255 at some pixel centre of the 8 x 8
// block whose first pixel centre is (x0, y0) (the test of warp_block_mask for
// one block).
__device__ __forceinline__ bool block_sees(const Rec& r, float x0, float y0) {
  const uint32_t e = __float_as_uint(r.c.w);
  const float hx = __half2float(__ushort_as_half((unsigned short)(e & 0xffffu)));
  const float hy = __half2float(__ushort_as_half((unsigned short)(e >> 16)));
  return r.a.x + hx >= x0 && r.a.x - hx <= x0 + 7.f && r.a.y + hy >= y0 && r.a.y - hy <= y0 + 7.f &&
         (!GS_EXACT_BLOCK_TEST || footprint_meets_block(r, x0, y0));
}

// 1: skip the reverse of a lane's first or second pixel when no lane of the
// warp blends the splat at that pixel.
#ifndef GS_BWD_SKIP_IDLE_ROW
#define GS_BWD_SKIP_IDLE_ROW 1
#endif
// A splat that at most this many lanes of a warp blend is added by those lanes
// one by one (each its own row of partial derivatives, as float4 atomics)
// instead of through the warp-wide reduction (0: always reduce).
#ifndef GS_BWD_SPARSE_LANES
#define GS_BWD_SPARSE_LANES 8
#endif
constexpr int kBwdSparseLanes = GS_BWD_SPARSE_LANES;
// Minimum resident CTAs per SM requested from the compiler for the reverse
// kernel (0: no request).
#ifndef GS_BWD_MIN_BLOCKS
#define GS_BWD_MIN_BLOCKS 7
#endif
#if GS_BWD_MIN_BLOCKS > 0
#define GS_BWD_BOUNDS(NT) __launch_bounds__(NT, (GS_BWD_MIN_BLOCKS * 128) / (NT))
#else
#define GS_BWD_BOUNDS(NT) __launch_bounds__(NT)
#endif

// Warp sums of v[0..31] delivered as quads: afterwards every lane L with
// (L & 3) == 0 holds in q[0..3] the warp-wide sums of v[L .. L+3].  Three
// reduce-scatter stages (lane bits 4, 3, 2) then a butterfly over bits 1, 0.
__device__ __forceinline__ void warp_reduce_quads32(float (&v)[32], float (&q)[4]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o >= 4; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; ++i) {
      const float send = up ? v[i] : v[i + o];
      const float keep = up ? v[i + o] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float x = v[i];
    x += __shfl_xor_sync(0xffffffffu, x, 1);
    x += __shfl_xor_sync(0xffffffffu, x, 2);
    q[i] = x;
  }
}
// Same for v[0..15] (slots 16..31 unused): lanes L < 16 with (L & 3) == 0 hold
// the sums of v[L .. L+3].
__device__ __forceinline__ void warp_reduce_quads16(float (&v)[32], float (&q)[4]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], 16);
#pragma unroll
  for (int o = 8; o >= 4; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; ++i) {
      const float send = up ? v[i] : v[i + o];
      const float keep = up ? v[i + o] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float x = v[i];
    x += __shfl_xor_sync(0xffffffffu, x, 1);
    x += __shfl_xor_sync(0xffffffffu, x, 2);
    q[i] = x;
  }
}

// Row stride (floats) of the per-view 2-D cotangents: 9 per stream, padded to
// whole float4s so that rows can be added and read as vectors.
__host__ __device__ constexpr int cot_stride(int streams) { return (9 * streams + 3) & ~3; }

// The reverse pass's workspace: a header, then the cotangent rows the reverse
// blend adds into.  They must be zero when the blend starts.  The projection
// reverse, which reads every row, leaves each row it read zero, and its last
// block records in the header that the first clear_floats floats are zero;
// the next call then clears nothing.  Any other header (a new or reused
// buffer, a call that stopped between the blend and the projection reverse)
// makes the next call clear the rows first; the blend marks the rows dirty
// when it starts.
struct CotHeader {
  uint64_t magic;         // kCotClear while clear_floats is valid
  uint64_t clear_floats;  // leading floats of the rows known to be zero
  uint32_t done_blocks;   // projection-reverse blocks finished in this call
};
constexpr uint64_t kCotClear = 0x9d2c5680a3b1f4e7ull;
constexpr size_t kCotHeaderBytes = 256;

// Zero the first 4 n4 floats of the rows unless the header says they are zero;
// reset the projection reverse's block count.
__global__ void cot_prepare_kernel(CotHeader* __restrict__ h, float4* __restrict__ cot, size_t n4) {
  const bool clear = h->magic == kCotClear && h->clear_floats >= 4 * n4;
  if (blockIdx.x == 0 && threadIdx.x == 0) h->done_blocks = 0;
  if (clear) return;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n4; k += (size_t)gridDim.x * blockDim.x)
    cot[k] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// End of a projection-reverse block: after every thread's zeroing stores, the
// last block to finish records that the first `floats` floats are zero.
__device__ __forceinline__ void cot_mark_clear(CotHeader* h, uint64_t floats) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0 && atomicAdd(&h->done_blocks, 1u) == gridDim.x - 1) {
    __threadfence();
    h->clear_floats = floats;
    h->magic = kCotClear;
  }
}

// 1: the reverse recovers T_i with the fast division intrinsic's reciprocal
// of 1 - alpha (at most 2 ulps off; 1 - alpha lies in [0.01, 1]) instead of
// the correctly rounded one, whose slower path also costs registers: about
// 2.5 ulps per recovered step instead of 1, which over the few hundred splats
// a pixel walks back stays orders of magnitude inside the gradient and
// curvature tolerances.
#ifndef GS_BWD_APPROX_RCP
#define GS_BWD_APPROX_RCP 1
#endif

// Reverse-pass state of one pixel: the cotangent dL/dC of each stream, the
// transmittance being recovered back to front, the colour suffix
// sum_{j>i} c_j a_j T_j, and the list position after its last blended splat.
template <int S>
struct BwdPixel {
  float w[S][3];
  float T, suf[3];
  float pxc, pyc;
  uint32_t nc;
};

// The reverse of one splat at one pixel: recover T_i = T_{i+1}/(1 - a),
// dC/da = c T_i - suffix/(1 - a), and store (FIRST) or add, for every stream,
// the pixel's terms of the splat's cotangent row in v: the moments
// (dx g, dy g, dx^2 g, dx dy g, dy^2 g) of g = dL/d(power), then dL/do,
// dL/d(r, g, b).  power = -(A dx^2 + C dy^2)/2 - B dx dy, so dL/dA = -M2/2,
// dL/dB = -M3, dL/dC = -M4/2, dL/dmx = -(A M0 + B M1), dL/dmy = -(B M0 + C M1).  A pixel the splat is not blended at passes alpha = G = oG = 0: its state
// stays as it is and it contributes exact zeros, so the pixels of a thread need
// no branches.  One reciprocal of 1 - a serves the four quotients.
template <int S, bool FIRST>
__device__ __forceinline__ void bwd_accumulate(BwdPixel<S>& p, const Rec& r, float dx, float dy, float G, float oG,
                                               float alpha, float (&v)[32]) {
#if GS_BWD_APPROX_RCP
  const float inv = __fdividef(1.f, 1.f - alpha);
#else
  const float inv = __frcp_rn(1.f - alpha);
#endif
  const float Ti = p.T * inv;
  const float rgb0 = r.b.z, rgb1 = r.b.w, rgb2 = r.c.x;
  const float da0 = rgb0 * Ti - p.suf[0] * inv;
  const float da1 = rgb1 * Ti - p.suf[1] * inv;
  const float da2 = rgb2 * Ti - p.suf[2] * inv;
  const float aT = alpha * Ti;
  p.suf[0] += rgb0 * aT;
  p.suf[1] += rgb1 * aT;
  p.suf[2] += rgb2 * aT;
  p.T = Ti;
  // a capped alpha has zero derivative: both of its factors vanish at once
  const bool capped = oG > kAlphaMax;
  const float ac = capped ? 0.f : alpha, Gc = capped ? 0.f : G;
  const float dxx = dx * dx, dxy = dx * dy, dyy = dy * dy;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const float ga = p.w[s][0] * da0 + p.w[s][1] * da1 + p.w[s][2] * da2;
    const float gp = ga * ac;  // dL/d(power)
    // the power's partials are linear in the conic, so the warp sums moments of
    // (dx, dy) and the projection's reverse pass applies the conic
    const float c[9] = {dx * gp, dy * gp, dxx * gp, dxy * gp, dyy * gp, ga * Gc,
                        p.w[s][0] * aT, p.w[s][1] * aT, p.w[s][2] * aT};
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      if constexpr (FIRST) v[9 * s + q] = c[q];
      else v[9 * s + q] += c[q];
    }
  }
}

template <int NU, bool GRAD, bool CB, int NT>
__global__ void GS_BWD_BOUNDS(NT) raster_bwd_kernel(
    const float4* __restrict__ rec, const uint32_t* __restrict__ vals, const uint32_t* __restrict__ ranges,
    const uint32_t* __restrict__ order, int n_pad, gs_frame fr, int Tx, int T, const float* __restrict__ image,
    const float* __restrict__ target,
    const float* __restrict__ final_T, const uint32_t* __restrict__ n_contrib, const float* __restrict__ image_tan,
    int loss_kind, float gn_floor, float inv_m, float* __restrict__ cot, float* __restrict__ loss_out,
    int loss_per_view, CotHeader* cot_hdr, const uint8_t* __restrict__ masks, int32_t* status) {
  constexpr int S = (GRAD ? 1 : 0) + NU;  // cotangent streams
  constexpr int NVP = cot_stride(S);      // padded row stride of their 9 S values
  static_assert(NVP <= 32, "streams");
  static_assert(NT <= 256, "s_loss holds one partial per warp, at most eight");
  extern __shared__ __align__(16) unsigned char smem[];
  const int nthr = blockDim.x, nwarps = nthr >> 5, batch = CB ? fr.batch : kBatchPerThread * nthr;
  constexpr int K = kBwdStages;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);                     // K phase barriers
  uint32_t* released = reinterpret_cast<uint32_t*>(smem + K * sizeof(uint64_t));  // K release counters
  Rec* buf = reinterpret_cast<Rec*>(smem + kBwdRingHdr);
  uint32_t* s_idx = reinterpret_cast<uint32_t*>(buf + K * batch);
  uint8_t* s_bits = reinterpret_cast<uint8_t*>(s_idx + K * batch);  // block masks of the staged records
  __shared__ uint32_t s_max;
  __shared__ int s_abort;
  __shared__ float s_loss[8];
  __shared__ int s_fill_use[kBwdStages];  // ring use of each stage's last fill (-1: none)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // the tile of this block: the heaviest tiles first when an order is given
  const int blk = order ? (int)min(__ldg(order + blockIdx.x), gridDim.x - 1) : (int)blockIdx.x;
  const int view = blk / T, tile = blk - view * T;
  const int ty = tile / Tx, tx = tile - ty * Tx;
  int lx, ly;
  pixel_of(tid, fr.tile_w, lx, ly);
  const size_t tslot = 2 * ((size_t)view * T + tile);
  const uint32_t start = ranges[tslot], list_len = ranges[tslot + 1] - start;
  const size_t HW = (size_t)fr.width * fr.height;
  // first pixel centre of this warp's 8 x 8 block
  const float wx0 = (float)(tx * fr.tile_w + (warp % (fr.tile_w >> 3)) * 8) + 0.5f;
  const float wy0 = (float)(ty * fr.tile_h + (warp / (fr.tile_w >> 3)) * 8) + 0.5f;

  // per-pixel cotangents dL/dC of each stream and the loss
  BwdPixel<S> pix[kPixPerThread];
  float lossp = 0.f;
#pragma unroll
  for (int q = 0; q < kPixPerThread; ++q) {
    BwdPixel<S>& p = pix[q];
    const int px = tx * fr.tile_w + lx, py = ty * fr.tile_h + ly + 4 * q;
    p.pxc = (float)px + 0.5f;
    p.pyc = (float)py + 0.5f;
    p.suf[0] = p.suf[1] = p.suf[2] = 0.f;
    p.T = 0.f;
    p.nc = 0;
#pragma unroll
    for (int st = 0; st < S; ++st) p.w[st][0] = p.w[st][1] = p.w[st][2] = 0.f;
    if (!(px < fr.width && py < fr.height)) continue;
    const size_t at0 = (size_t)py * fr.width + px;
    p.T = final_T[(size_t)view * HW + at0];
    p.nc = n_contrib[(size_t)view * HW + at0];
    if (loss_kind == GS_LOSS_COTANGENT) {  // the caller's cotangent images, one per stream
#pragma unroll
      for (int st = 0; st < S; ++st)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) p.w[st][ch] = target[(((size_t)st * fr.n_views + view) * 3 + ch) * HW + at0];
      continue;
    }
    if (loss_kind == GS_LOSS_WEIGHTED) {  // dL/dC (gradient stream), then the weights of w . J z_k
      const float* wimg = target + (GRAD ? (size_t)fr.n_views * 3 * HW : 0);
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        if constexpr (GRAD) p.w[0][ch] = target[((size_t)view * 3 + ch) * HW + at0];
        const float wv = wimg[((size_t)view * 3 + ch) * HW + at0];
#pragma unroll
        for (int k = 0; k < NU; ++k)
          p.w[(GRAD ? 1 : 0) + k][ch] = wv * image_tan[(((size_t)k * fr.n_views + view) * 3 + ch) * HW + at0];
      }
      continue;
    }
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      const size_t at = ((size_t)view * 3 + ch) * HW + at0;
      const float r = image[at] - target[at];
      const float ar = fabsf(r);
      float lam;
      if (loss_kind == GS_LOSS_L1) {
        lossp += 0.5f * inv_m * ar;
        lam = 0.25f / fmaxf(ar, gn_floor);
      } else {
        lossp += 0.5f * inv_m * r * r;
        lam = 1.f;
      }
      if constexpr (GRAD) p.w[0][ch] = (loss_kind == GS_LOSS_L1) ? (0.5f * inv_m) * ((r > 0.f) - (r < 0.f)) : inv_m * r;
#pragma unroll
      for (int k = 0; k < NU; ++k)
        p.w[(GRAD ? 1 : 0) + k][ch] = inv_m * lam * image_tan[(((size_t)k * fr.n_views + view) * 3 + ch) * HW + at0];
    }
  }
  if (tid == 0) {
    if (blockIdx.x == 0) cot_hdr->clear_floats = 0;  // the rows are being added into
    s_max = 0;
    // a stage wait that ran out in an earlier block: skip the list walk
    s_abort = status ? (*(volatile int32_t*)status & GS_FLAG_TIMEOUT) : 0;
    for (int k = 0; k < K; ++k) {
      mbar_init(&full[k], 1);
      released[k] = 0;
      s_fill_use[k] = -1;
    }
    fence_mbar_init();
  }
  __syncthreads();
  const uint32_t nc_thread = max(pix[0].nc, pix[1].nc);
  if (nc_thread) atomicMax(&s_max, nc_thread);
  const uint32_t warp_nc = __reduce_max_sync(0xffffffffu, nc_thread);  // list positions this warp still needs
  // objective: warp then block reduction, one atomic per CTA
  if (loss_out) {
    float lsum = lossp;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0) s_loss[tid >> 5] = lsum;
  }
  __syncthreads();
  if (loss_out && tid == 0) {
    float tot = 0.f;
    for (int k = 0; k < nwarps; ++k) tot += s_loss[k];
    atomicAdd(loss_out + (loss_per_view ? view : 0), tot);
  }
  const int n = s_abort ? 0 : (int)min(s_max, list_len);  // n_contrib never exceeds the tile's list
  const int nb = (n + batch - 1) / batch;
  // batch b is use u = nb - 1 - b of the ring: stage u % K, its (u / K)-th fill
  for (int u = warp; u < min(K, nb); u += nwarps)
    stage_batch_warp(u, u, nb - 1 - u, batch, start, n, view, n_pad, vals, rec, masks, buf, s_idx, s_bits, full,
                     s_fill_use);
  bool ok = true;
  for (int u = 0; u < nb; ++u) {
    const int st = u % K, b = nb - 1 - u;
    // every lane waits (bounded) for the stage's phase: each acquires the copies
    // and indices.  A warp whose wait ran out stops at once: it releases no
    // further stage, so no later round completes and nothing is refilled
    // behind it; the other warps run into their own bounded waits.
    const bool landed = mbar_wait_bounded(&full[st], (uint32_t)((u / K) & 1), status);
    ok = __all_sync(0xffffffffu, landed) != 0;
    if (!ok) break;
    const int cnt = min(batch, n - b * batch);
    const Rec* bb = buf + st * batch;
    // the warp walks, back to front, only the splats its block can see (the
    // forward pass's mask bit when given, else the same footprint test) and
    // that lie before its last contributor: one ballot per 32 splats
    const uint8_t* sb = s_bits + st * batch;
    for (int j0 = ((cnt - 1) & ~31); (uint32_t)(b * batch) < warp_nc && j0 >= 0; j0 -= 32) {
      const int jl = j0 + lane;
      uint32_t bits = __ballot_sync(
          0xffffffffu, jl < cnt && (uint32_t)(b * batch + jl) < warp_nc &&
                           (masks ? ((sb[jl] >> warp) & 1u) != 0 : block_sees(bb[jl], wx0, wy0)));
      while (bits) {
        const int hb = 31 - __clz(bits);
        bits &= ~(1u << hb);
        const int j = j0 + hb;
        const uint32_t pos = (uint32_t)(b * batch + j);
        const Rec r = bb[j];
        bool on[kPixPerThread];
        float dx[kPixPerThread], dy[kPixPerThread], G[kPixPerThread], oG[kPixPerThread], alpha[kPixPerThread];
#pragma unroll
        for (int q = 0; q < kPixPerThread; ++q) {
          dx[q] = __fsub_rn(r.a.x, pix[q].pxc);
          dy[q] = __fsub_rn(r.a.y, pix[q].pyc);
          const float power = splat_power(r, dx[q], dy[q]);
          G[q] = __expf(power);
          oG[q] = __fmul_rn(r.b.y, G[q]);
          alpha[q] = fminf(kAlphaMax, oG[q]);
          on[q] = pos < pix[q].nc && power <= 0.f && alpha[q] >= kAlphaMin;
          if (!on[q]) G[q] = oG[q] = alpha[q] = 0.f;
        }
        const uint32_t act = __ballot_sync(0xffffffffu, on[0] || on[1]);  // lanes that blend the splat
        if (!act) continue;
        float v[32];
#if GS_BWD_SKIP_IDLE_ROW
        // a pixel row of the block (the lanes' first or second pixels) that no
        // lane blends the splat at adds exact zeros and keeps its state: skip it
        const bool any0 = __any_sync(0xffffffffu, on[0]), any1 = __any_sync(0xffffffffu, on[1]);
        if (any0) {
          bwd_accumulate<S, true>(pix[0], r, dx[0], dy[0], G[0], oG[0], alpha[0], v);
          if (any1) bwd_accumulate<S, false>(pix[1], r, dx[1], dy[1], G[1], oG[1], alpha[1], v);
        } else {
          bwd_accumulate<S, true>(pix[1], r, dx[1], dy[1], G[1], oG[1], alpha[1], v);
        }
#else
        bwd_accumulate<S, true>(pix[0], r, dx[0], dy[0], G[0], oG[0], alpha[0], v);
        bwd_accumulate<S, false>(pix[1], r, dx[1], dy[1], G[1], oG[1], alpha[1], v);
#endif
#pragma unroll
        for (int q = 9 * S; q < 32; ++q) v[q] = 0.f;
        const uint32_t gi = s_idx[st * batch + j];
        float* dst = cot + ((size_t)view * n_pad + gi) * NVP;
        if (__popc(act) <= kBwdSparseLanes) {
          // few lanes blend the splat: each adds its own row instead of the
          // warp-wide reduction (the other lanes' rows are zero)
          if (on[0] || on[1]) {
#pragma unroll
            for (int q = 0; q < NVP; q += 4)
              atomicAdd(reinterpret_cast<float4*>(dst + q), make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]));
          }
          continue;
        }
        float qs[4];
        if constexpr (NVP <= 16) warp_reduce_quads16(v, qs);
        else warp_reduce_quads32(v, qs);
        if ((lane & 3) == 0 && lane < NVP && (qs[0] != 0.f || qs[1] != 0.f || qs[2] != 0.f || qs[3] != 0.f))
          atomicAdd(reinterpret_cast<float4*>(dst + lane), make_float4(qs[0], qs[1], qs[2], qs[3]));
      }
    }
    // release the stage: the warp's reads of it are ordered before its count,
    // and the last warp to count it, ordered after all counts, refills it
    __syncwarp();
    uint32_t last = 0;
    if (lane == 0) {
      __threadfence_block();
      last = atomicAdd(&released[st], 1u) == (uint32_t)(nwarps - 1);
      if (last) {
        released[st] = 0;
        __threadfence_block();
      }
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (last && u + K < nb)
      stage_batch_warp(st, u + K, nb - 1 - (u + K), batch, start, n, view, n_pad, vals, rec, masks, buf, s_idx,
                       s_bits, full, s_fill_use);
  }
  // Drain after a failed wait: a stage is refilled only by a warp that saw its
  // previous fill land, so each stage has at most one fill in flight, its last.
  // One thread per stage waits (bounded) for that fill, so that no bulk copy is
  // still writing into this block's shared memory, or completing on its
  // barrier, when the block exits.  Without a failure every fill has landed.
  if (__syncthreads_or(!ok) && tid < K && s_fill_use[tid] >= 0)
    mbar_wait_bounded(&full[tid], (uint32_t)((s_fill_use[tid] / K) & 1), status);
}

// ------------------------------------------------ projection reverse pass
// Reverse pass of the EWA projection and SH colour for one Gaussian, summed over
// views.  The chain rule, written out:
//   conic = Sigma'^-1:   dA/da = -c^2/det^2, dA/db = 2bc/det^2, dA/dc = 1/det - ac/det^2,
//                        dB/da = bc/det^2, dB/db = -1/det - 2b^2/det^2, dB/dc = ab/det^2,
//                        dC/da = 1/det - ac/det^2, dC/db = 2ab/det^2, dC/dc = -a^2/det^2
//   Sigma' = J Sc J^T:   dSc = J^T Gs J, dJ = 2 Gs J Sc, Gs = [[ga, gb/2], [gb/2, gc]]
//   J(t):                the slope clamp cuts the t_x (t_y) path, J02 = -fx uc / tz
//   Sc = W Sigma W^T:    dSigma = W^T dSc W = (W^T J^T) Gs (J W), summed as the 6
//                        entries of a symmetric matrix from a0 = W^T j0, a1 = W^T j1
//                        (j0, j1 the rows of J);   mean2D(t) and t = W mu + t_w
//   Sigma = M M^T:       dM = 2 dSigma M, M = R diag(s), s = exp(log s)
//   R(q / |q|):          dq = (dqn - qn (qn . dqn)) / |q|
//   colour:              dSH_k = Y_k dc (0 where clamped), dmu += P_perp grad_Y . (sum sh dc) / |d|
// One thread per Gaussian.  A first pass over the views computes each view's
// geometry once and applies it to every cotangent stream (geometric rows); a
// second pass per stream accumulates the SH rows, reusing the clamp decisions
// recorded in the first.  The first pass also keeps the clamped colour
// cotangents of the first kStashViews views in shared memory, so the second
// pass reads them there instead of from L2.  The probe streams are combined into
// hz = (1/nu) sum_k z_k . (G z_k).
constexpr int kPbwdThreads = 128;
// Minimum resident CTAs per SM requested for the projection reverse (0: none).
#ifndef GS_PBWD_MIN_BLOCKS
#define GS_PBWD_MIN_BLOCKS 3
#endif
#if GS_PBWD_MIN_BLOCKS > 0
#define GS_PBWD_BOUNDS __launch_bounds__(kPbwdThreads, GS_PBWD_MIN_BLOCKS)
#else
#define GS_PBWD_BOUNDS __launch_bounds__(kPbwdThreads)
#endif
constexpr int kClampViews = 21;  // clamp bits kept for the first 21 views (3 per view)
constexpr int kStashViews = 8;   // views whose colour cotangents pass 2 reads from shared memory

// dynamic shared memory of the projection reverse: min(V, kStashViews) x 3S x kPbwdThreads floats
__host__ __device__ constexpr size_t pbwd_stash_bytes(int n_views, int streams) {
  return (size_t)(n_views < kStashViews ? n_views : kStashViews) * 3 * streams * kPbwdThreads * sizeof(float);
}

struct ViewGeom {
  float Rc[3][3], tc[3], fx, fy;
};

__device__ __forceinline__ void load_view(const gs_camera* cam, ViewGeom& v) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) v.Rc[a][b] = cam->viewmat[4 * a + b];
    v.tc[a] = cam->viewmat[4 * a + 3];
  }
  v.fx = cam->fx;
  v.fy = cam->fy;
}

// Unit view direction and distance from the camera centre to mu.
__device__ __forceinline__ void view_direction(const ViewGeom& v, const float mu[3], float d[3], float& dn) {
  float cp[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) cp[q] = -(v.Rc[0][q] * v.tc[0] + v.Rc[1][q] * v.tc[1] + v.Rc[2][q] * v.tc[2]);
  const float d0 = mu[0] - cp[0], d1 = mu[1] - cp[1], d2 = mu[2] - cp[2];
  dn = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
  d[0] = d0 / dn;
  d[1] = d1 / dn;
  d[2] = d2 / dn;
}

// Column i (of n Gaussians, parameter pitch n_pad) summed over views cams[0..V),
// its cotangent row of view v at (v * cot_pitch + i) * NVP of cot.  Called by
// every thread of a kPbwdThreads block (the SH staging is block-wide).
template <int DEG, int NU, bool GRAD>
__device__ __forceinline__ void project_bwd_column(const float* __restrict__ P, int n, int n_pad, int i,
                                                   const gs_camera* __restrict__ cams, int V, gs_frame fr,
                                                   float* __restrict__ cot, int cot_pitch, ProbeArg pa,
                                                   float* __restrict__ grad, float* __restrict__ hz) {
  constexpr int S = (GRAD ? 1 : 0) + NU;
  constexpr int NVP = cot_stride(S);
  constexpr int K = (DEG + 1) * (DEG + 1);
  // the block's SH coefficients, staged once and read per view from shared
  // memory (volatile: re-read, not held in registers across the view loops)
  __shared__ float s_sh[3 * K][kPbwdThreads];
  for (int r = 0; r < 3 * K; ++r) s_sh[r][threadIdx.x] = i < n ? P[(size_t)(kRowSH + r) * n_pad + i] : 0.f;
  __syncthreads();
  const volatile float* vsh = &s_sh[0][0];
  auto sh_of = [&](int k, int ch) { return vsh[(3 * k + ch) * kPbwdThreads + threadIdx.x]; };
  // colour cotangents (0 where clamped) of views v < kStashViews, one column per thread
  extern __shared__ float s_pbwd_stash[];
  auto stash = [&](int v, int j) -> float& { return s_pbwd_stash[(v * 3 * S + j) * kPbwdThreads + threadIdx.x]; };
  if (i >= n) return;
  const uint64_t seed = pa.seed;
  const int64_t step = NU > 0 ? probe_step(pa) : 0;
  auto ld = [&](int r) { return __ldg(P + (size_t)r * n_pad + i); };
  const float mu[3] = {ld(0), ld(1), ld(2)};
  float qx = ld(6), qy = ld(7), qz = ld(8), qw = ld(9);
  const float qlen = sqrtf(qx * qx + qy * qy + qz * qz + qw * qw);
  qx /= qlen; qy /= qlen; qz /= qlen; qw /= qlen;
  float R[3][3];
  R[0][0] = 1.f - 2.f * (qy * qy + qz * qz);
  R[0][1] = 2.f * (qx * qy - qw * qz);
  R[0][2] = 2.f * (qx * qz + qw * qy);
  R[1][0] = 2.f * (qx * qy + qw * qz);
  R[1][1] = 1.f - 2.f * (qz * qz + qx * qx);
  R[1][2] = 2.f * (qy * qz - qw * qx);
  R[2][0] = 2.f * (qx * qz - qw * qy);
  R[2][1] = 2.f * (qy * qz + qw * qx);
  R[2][2] = 1.f - 2.f * (qx * qx + qy * qy);
  float sc[3], M[3][3], Sg[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) sc[a] = expf(ld(3 + a));
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) M[a][b] = R[a][b] * sc[b];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) Sg[a][b] = M[a][0] * M[b][0] + M[a][1] * M[b][1] + M[a][2] * M[b][2];
  const float opac = 1.f / (1.f + expf(-ld(10)));
  const float dsig = opac * (1.f - opac);

  // ---- pass 1: geometric rows of every stream
  // g_S: dL/dSigma, symmetric, entries (0,0) (0,1) (0,2) (1,1) (1,2) (2,2)
  constexpr int kSymP[6] = {0, 0, 0, 1, 1, 2}, kSymQ[6] = {0, 1, 2, 1, 2, 2};
  float g_mu[S][3], g_S[S][6], g_ol[S];
#pragma unroll
  for (int st = 0; st < S; ++st) {
    g_ol[st] = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) g_mu[st][a] = 0.f;
#pragma unroll
    for (int e = 0; e < 6; ++e) g_S[st][e] = 0.f;
  }
  uint64_t clamp_bits = 0;  // bit 3 v + c: colour channel c clamped at 0 in view v (v < kClampViews)
  uint64_t read_rows = 0;   // bit v: the row of view v held a nonzero value (cleared at the end; v >= 64 always)
#pragma unroll 1
  for (int v = 0; v < V; ++v) {
    float c[NVP];
    bool any = false;
    const float4* row4 = reinterpret_cast<const float4*>(cot + ((size_t)v * cot_pitch + i) * NVP);
#pragma unroll
    for (int q = 0; q < NVP / 4; ++q) {
      const float4 x4 = row4[q];
      c[4 * q + 0] = x4.x; c[4 * q + 1] = x4.y; c[4 * q + 2] = x4.z; c[4 * q + 3] = x4.w;
      any = any || x4.x != 0.f || x4.y != 0.f || x4.z != 0.f || x4.w != 0.f;
    }
    if (v < 64) read_rows |= (uint64_t)any << v;
    if (!any) {
      if (v < kStashViews) {
#pragma unroll
        for (int j = 0; j < 3 * S; ++j) stash(v, j) = 0.f;
      }
      continue;
    }
    ViewGeom vg;
    load_view(cams + v, vg);
    const float fx = vg.fx, fy = vg.fy;
    float t[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) t[a] = vg.Rc[a][0] * mu[0] + vg.Rc[a][1] * mu[1] + vg.Rc[a][2] * mu[2] + vg.tc[a];
    float Sc[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float tmp[3];
#pragma unroll
      for (int b = 0; b < 3; ++b) tmp[b] = vg.Rc[a][0] * Sg[0][b] + vg.Rc[a][1] * Sg[1][b] + vg.Rc[a][2] * Sg[2][b];
#pragma unroll
      for (int b = 0; b < 3; ++b) Sc[a][b] = tmp[0] * vg.Rc[b][0] + tmp[1] * vg.Rc[b][1] + tmp[2] * vg.Rc[b][2];
    }
    const float limx = kSlopeClamp * 0.5f * (float)fr.width / fx;
    const float limy = kSlopeClamp * 0.5f * (float)fr.height / fy;
    const float itz = 1.f / t[2];
    const float u = t[0] * itz, vv = t[1] * itz;
    const bool clx = u < -limx || u > limx, cly = vv < -limy || vv > limy;
    const float uc = fminf(fmaxf(u, -limx), limx), vc = fminf(fmaxf(vv, -limy), limy);
    const float J00 = fx * itz, J02 = -fx * uc * itz, J11 = fy * itz, J12 = -fy * vc * itz;
    const float a = J00 * J00 * Sc[0][0] + 2.f * J00 * J02 * Sc[0][2] + J02 * J02 * Sc[2][2] + kDilation;
    const float bb = J00 * J11 * Sc[0][1] + J00 * J12 * Sc[0][2] + J02 * J11 * Sc[1][2] + J02 * J12 * Sc[2][2];
    const float cc = J11 * J11 * Sc[1][1] + 2.f * J11 * J12 * Sc[1][2] + J12 * J12 * Sc[2][2] + kDilation;
    const float det = a * cc - bb * bb;
    const float idet = 1.f / det, id2 = idet * idet;
    // rows of J taken back to world axes: a0 = W^T j0, a1 = W^T j1
    float a0[3], a1[3];
#pragma unroll
    for (int p2 = 0; p2 < 3; ++p2) {
      a0[p2] = vg.Rc[0][p2] * J00 + vg.Rc[2][p2] * J02;
      a1[p2] = vg.Rc[1][p2] * J11 + vg.Rc[2][p2] * J12;
    }
    float JS0[3], JS1[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      JS0[q] = J00 * Sc[0][q] + J02 * Sc[2][q];
      JS1[q] = J11 * Sc[1][q] + J12 * Sc[2][q];
    }
    const float itz2 = itz * itz, itz3 = itz2 * itz;
    const float dJ02_dtx = clx ? 0.f : -fx * itz2, dJ12_dty = cly ? 0.f : -fy * itz2;
    const float dJ02_dtz = clx ? fx * uc * itz2 : 2.f * fx * t[0] * itz3;
    const float dJ12_dtz = cly ? fy * vc * itz2 : 2.f * fy * t[1] * itz3;
    // conic of this view, to turn the blend's moments into dL/d(mx, my, A, B, C)
    const float cA = cc * idet, cB = -bb * idet, cCc = a * idet;
#pragma unroll
    for (int st = 0; st < S; ++st) {
      const float* mo = c + 9 * st;
      const float cs[5] = {-(cA * mo[0] + cB * mo[1]), -(cB * mo[0] + cCc * mo[1]), -0.5f * mo[2], -mo[3],
                           -0.5f * mo[4]};
      const float gA = cs[2], gB = cs[3], gC = cs[4];
      const float ga = gA * (-cc * cc * id2) + gB * (bb * cc * id2) + gC * (idet - a * cc * id2);
      const float gb = gA * (2.f * bb * cc * id2) + gB * (-idet - 2.f * bb * bb * id2) + gC * (2.f * a * bb * id2);
      const float gc = gA * (idet - a * cc * id2) + gB * (a * bb * id2) + gC * (-a * a * id2);
      const float gJ00 = 2.f * (ga * JS0[0] + 0.5f * gb * JS1[0]);
      const float gJ02 = 2.f * (ga * JS0[2] + 0.5f * gb * JS1[2]);
      const float gJ11 = 2.f * (0.5f * gb * JS0[1] + gc * JS1[1]);
      const float gJ12 = 2.f * (0.5f * gb * JS0[2] + gc * JS1[2]);
      float gt[3];
      gt[0] = cs[0] * fx * itz + gJ02 * dJ02_dtx;
      gt[1] = cs[1] * fy * itz + gJ12 * dJ12_dty;
      gt[2] = -cs[0] * fx * t[0] * itz2 - cs[1] * fy * t[1] * itz2 - gJ00 * fx * itz2 - gJ11 * fy * itz2 +
              gJ02 * dJ02_dtz + gJ12 * dJ12_dtz;
#pragma unroll
      for (int q = 0; q < 3; ++q) g_mu[st][q] += vg.Rc[0][q] * gt[0] + vg.Rc[1][q] * gt[1] + vg.Rc[2][q] * gt[2];
      // dSigma += ga a0 a0^T + gb/2 (a0 a1^T + a1 a0^T) + gc a1 a1^T = u a0^T + w a1^T
      {
        const float hb = 0.5f * gb;
        float u[3], w[3];
#pragma unroll
        for (int p2 = 0; p2 < 3; ++p2) {
          u[p2] = ga * a0[p2] + hb * a1[p2];
          w[p2] = hb * a0[p2] + gc * a1[p2];
        }
#pragma unroll
        for (int e = 0; e < 6; ++e) g_S[st][e] += u[kSymP[e]] * a0[kSymQ[e]] + w[kSymP[e]] * a1[kSymQ[e]];
      }
      g_ol[st] += mo[5] * dsig;
    }
    // colour: clamp decisions, and the dependence of colour on mu through the view direction
    float d[3], dn;
    view_direction(vg, mu, d, dn);
    float Y[K];
    sh_basis<DEG>(d[0], d[1], d[2], Y);
    // per channel: the raw colour (its clamp decision) and, for the colour's
    // dependence on mu, the direction gradient of sum_k sh_k Y_k; the SH
    // coefficients come from the staged copy instead of registers
    bool clamped[3];
    float gdc[3][3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      float shc[K];
#pragma unroll
      for (int k = 0; k < K; ++k) shc[k] = sh_of(k, ch);
      float raw = 0.5f;
#pragma unroll
      for (int k = 0; k < K; ++k) raw += Y[k] * shc[k];
      clamped[ch] = raw < 0.f;
      if (clamped[ch] && v < kClampViews) clamp_bits |= 1ull << (3 * v + ch);
      if constexpr (DEG > 0) sh_basis_grad<DEG>(d[0], d[1], d[2], shc, gdc[ch]);
    }
    if (v < kStashViews) {
#pragma unroll
      for (int st = 0; st < S; ++st)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) stash(v, 3 * st + ch) = clamped[ch] ? 0.f : c[9 * st + 6 + ch];
    }
    if constexpr (DEG > 0) {
#pragma unroll
      for (int st = 0; st < S; ++st) {
        float gcol[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) gcol[ch] = clamped[ch] ? 0.f : c[9 * st + 6 + ch];
        float gd[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) gd[q] = gcol[0] * gdc[0][q] + gcol[1] * gdc[1][q] + gcol[2] * gdc[2][q];
        const float dot = gd[0] * d[0] + gd[1] * d[1] + gd[2] * d[2];
#pragma unroll
        for (int q = 0; q < 3; ++q) g_mu[st][q] += (gd[q] - d[q] * dot) / dn;
      }
    }
  }

  // ---- geometric rows: Sigma = M M^T, M = R diag(s); R(q / |q|)
  const float qn[4] = {qx, qy, qz, qw};
  float hz_geo[kRowSH];
#pragma unroll
  for (int r = 0; r < kRowSH; ++r) hz_geo[r] = 0.f;
  const float inv_nu = NU > 0 ? 1.f / (float)NU : 0.f;
#pragma unroll
  for (int st = 0; st < S; ++st) {
    const float gS[3][3] = {{g_S[st][0], g_S[st][1], g_S[st][2]},
                            {g_S[st][1], g_S[st][3], g_S[st][4]},
                            {g_S[st][2], g_S[st][4], g_S[st][5]}};
    float gM[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) gM[a][b] = 2.f * (gS[a][0] * M[0][b] + gS[a][1] * M[1][b] + gS[a][2] * M[2][b]);
    float rowv[kRowSH];
    float gR[3][3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      rowv[3 + b] = (gM[0][b] * R[0][b] + gM[1][b] * R[1][b] + gM[2][b] * R[2][b]) * sc[b];
#pragma unroll
      for (int a = 0; a < 3; ++a) gR[a][b] = gM[a][b] * sc[b];
    }
    const float x = qx, y = qy, z = qz, ww = qw;
    float gq[4];
    gq[0] = 2.f * y * gR[0][1] + 2.f * z * gR[0][2] + 2.f * y * gR[1][0] - 4.f * x * gR[1][1] - 2.f * ww * gR[1][2] +
            2.f * z * gR[2][0] + 2.f * ww * gR[2][1] - 4.f * x * gR[2][2];
    gq[1] = -4.f * y * gR[0][0] + 2.f * x * gR[0][1] + 2.f * ww * gR[0][2] + 2.f * x * gR[1][0] + 2.f * z * gR[1][2] -
            2.f * ww * gR[2][0] + 2.f * z * gR[2][1] - 4.f * y * gR[2][2];
    gq[2] = -4.f * z * gR[0][0] - 2.f * ww * gR[0][1] + 2.f * x * gR[0][2] + 2.f * ww * gR[1][0] - 4.f * z * gR[1][1] +
            2.f * y * gR[1][2] + 2.f * x * gR[2][0] + 2.f * y * gR[2][1];
    gq[3] = -2.f * z * gR[0][1] + 2.f * y * gR[0][2] + 2.f * z * gR[1][0] - 2.f * x * gR[1][2] - 2.f * y * gR[2][0] +
            2.f * x * gR[2][1];
    const float qd = gq[0] * x + gq[1] * y + gq[2] * z + gq[3] * ww;
#pragma unroll
    for (int a = 0; a < 3; ++a) rowv[a] = g_mu[st][a];
#pragma unroll
    for (int cq = 0; cq < 4; ++cq) rowv[6 + cq] = (gq[cq] - qn[cq] * qd) / qlen;
    rowv[10] = g_ol[st];
    if (GRAD && st == 0) {
#pragma unroll
      for (int r = 0; r < kRowSH; ++r) grad[(size_t)r * n_pad + i] = rowv[r];
    } else {
      const int k = st - (GRAD ? 1 : 0);
      const uint64_t zneg = probe_signs(seed, step, k, (uint64_t)i, kRowSH + 3 * K);
#pragma unroll
      for (int r = 0; r < kRowSH; ++r) {
        const bool neg = (zneg >> r) & 1ull;
        hz_geo[r] += (neg ? -rowv[r] : rowv[r]) * inv_nu;
      }
    }
  }
  if constexpr (NU > 0) {
#pragma unroll
    for (int r = 0; r < kRowSH; ++r) hz[(size_t)r * n_pad + i] = hz_geo[r];
  }

  // ---- pass 2: SH rows, dSH_k = sum_v Y_k(d_v) dc_v.  The gradient stream
  // alone; two probe streams in one walk over the views: z1 . G1 + z2 . G2 =
  // z1 . (G1 + (z1 z2) G2), so the sums of Y (dc1 + dc2) and Y (dc1 - dc2) are
  // kept and each row's sign product picks one.
  // colour cotangent of view v, stream st (clamps applied for v < kStashViews)
  auto colour_cot = [&](int v, int st, float (&g)[3]) {
    if (v < kStashViews) {
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) g[ch] = stash(v, 3 * st + ch);
    } else {
      const float* cv = cot + ((size_t)v * cot_pitch + i) * NVP + 9 * st + 6;
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) g[ch] = cv[ch];
    }
  };
  // basis of view v and its clamp decisions (true: channel clamped at 0)
  auto view_basis = [&](int v, float (&Y)[K], bool (&cl)[3]) {
    ViewGeom vg;
    load_view(cams + v, vg);
    float d[3], dn;
    view_direction(vg, mu, d, dn);
    sh_basis<DEG>(d[0], d[1], d[2], Y);
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      if (v < kStashViews) {
        cl[ch] = false;  // already applied
      } else if (v < kClampViews) {
        cl[ch] = (clamp_bits >> (3 * v + ch)) & 1ull;
      } else {
        float raw = 0.5f;
#pragma unroll
        for (int k = 0; k < K; ++k) raw += Y[k] * sh_of(k, ch);
        cl[ch] = raw < 0.f;
      }
    }
  };
  auto sh_rows_single = [&](int st) {
    float g_sh[K][3];
#pragma unroll
    for (int k = 0; k < K; ++k) g_sh[k][0] = g_sh[k][1] = g_sh[k][2] = 0.f;
#pragma unroll 1
    for (int v = 0; v < V; ++v) {
      float gcol[3];
      colour_cot(v, st, gcol);
      if (gcol[0] == 0.f && gcol[1] == 0.f && gcol[2] == 0.f) continue;
      float Y[K];
      bool cl[3];
      view_basis(v, Y, cl);
#pragma unroll
      for (int ch = 0; ch < 3; ++ch)
        if (cl[ch]) gcol[ch] = 0.f;
#pragma unroll
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) g_sh[k][ch] += Y[k] * gcol[ch];
    }
    if (GRAD && st == 0) {
#pragma unroll
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) grad[(size_t)(kRowSH + 3 * k + ch) * n_pad + i] = g_sh[k][ch];
    } else {
      const uint64_t zneg = probe_signs(seed, step, st - (GRAD ? 1 : 0), (uint64_t)i, kRowSH + 3 * K);
#pragma unroll
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
          const int r = kRowSH + 3 * k + ch;
          const bool neg = (zneg >> r) & 1ull;
          hz[(size_t)r * n_pad + i] = (neg ? -g_sh[k][ch] : g_sh[k][ch]) * inv_nu;
        }
    }
  };
  if constexpr (GRAD) sh_rows_single(0);
  if constexpr (NU == 1) sh_rows_single(GRAD ? 1 : 0);
  if constexpr (NU == 2) {
    constexpr int s1 = GRAD ? 1 : 0, s2 = s1 + 1;
    float sp[K][3], sm[K][3];  // sums of Y (dc1 + dc2) and Y (dc1 - dc2)
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) sp[k][ch] = sm[k][ch] = 0.f;
#pragma unroll 1
    for (int v = 0; v < V; ++v) {
      float g1[3], g2[3];
      colour_cot(v, s1, g1);
      colour_cot(v, s2, g2);
      if (g1[0] == 0.f && g1[1] == 0.f && g1[2] == 0.f && g2[0] == 0.f && g2[1] == 0.f && g2[2] == 0.f) continue;
      float Y[K];
      bool cl[3];
      view_basis(v, Y, cl);
      float gp[3], gm[3];
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        gp[ch] = cl[ch] ? 0.f : g1[ch] + g2[ch];
        gm[ch] = cl[ch] ? 0.f : g1[ch] - g2[ch];
      }
#pragma unroll
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
          sp[k][ch] += Y[k] * gp[ch];
          sm[k][ch] += Y[k] * gm[ch];
        }
    }
    const uint64_t zn1 = probe_signs(seed, step, 0, (uint64_t)i, kRowSH + 3 * K);
    const uint64_t zn2 = probe_signs(seed, step, 1, (uint64_t)i, kRowSH + 3 * K);
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        const int r = kRowSH + 3 * k + ch;
        const bool n1 = (zn1 >> r) & 1ull, same = ((zn1 ^ zn2) >> r & 1ull) == 0;
        const float val = same ? sp[k][ch] : sm[k][ch];
        hz[(size_t)r * n_pad + i] = (n1 ? -val : val) * inv_nu;
      }
  }
  // leave the rows read above zero for the next call (CotHeader)
  for (int v = 0; v < V; ++v) {
    if (v < 64 && !((read_rows >> v) & 1ull)) continue;
    float4* row4 = reinterpret_cast<float4*>(cot + ((size_t)v * cot_pitch + i) * NVP);
#pragma unroll
    for (int q = 0; q < NVP / 4; ++q) row4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

template <int DEG, int NU, bool GRAD>
__global__ void GS_PBWD_BOUNDS project_bwd_kernel(const float* __restrict__ P, int n, int n_pad,
                                                  const gs_camera* __restrict__ cams, gs_frame fr,
                                                  float* __restrict__ cot, ProbeArg pa, float* __restrict__ grad,
                                                  float* __restrict__ hz, CotHeader* cot_hdr, uint64_t cot_floats) {
  const int i = blockIdx.x * kPbwdThreads + threadIdx.x;
  project_bwd_column<DEG, NU, GRAD>(P, n, n_pad, i, cams, fr.n_views, fr, cot, n_pad, pa, grad, hz);
  cot_mark_clear(cot_hdr, cot_floats);
}

// A batch: item b's share of the grid takes its columns through the reverse of
// its own projection, from its slot of the cotangents (pitch cot_pitch), with
// its own probe step, into its own gradient and Hutchinson rows.
template <int DEG, int NU, bool GRAD>
__global__ void GS_PBWD_BOUNDS project_bwd_batch_kernel(BatchArg ba, gs_frame fr, float* __restrict__ cot,
                                                        int cot_pitch, ProbeArg pa, CotHeader* cot_hdr,
                                                        uint64_t cot_floats) {
  constexpr int NVP = cot_stride((GRAD ? 1 : 0) + NU);
  const int b = batch_item(ba, (int)blockIdx.x);
  const int i = ((int)blockIdx.x - ba.first_block[b]) * kPbwdThreads + threadIdx.x;
  pa.t = ba.t[b];
  pa.t_dev = nullptr;
  project_bwd_column<DEG, NU, GRAD>(ba.P[b], ba.n[b], ba.n_pad[b], i, ba.cam[b], 1, fr,
                                    cot + (size_t)b * cot_pitch * NVP, cot_pitch, pa, ba.grad[b], ba.hz[b]);
  cot_mark_clear(cot_hdr, cot_floats);
}

// ------------------------------------------------------------------ host side
struct TileGrid {
  int Tx, Ty, T;
};
TileGrid tile_grid(gs_frame fr) {
  TileGrid g;
  g.Tx = (fr.width + fr.tile_w - 1) / fr.tile_w;
  g.Ty = (fr.height + fr.tile_h - 1) / fr.tile_h;
  g.T = g.Tx * g.Ty;
  return g;
}

template <class F>
cudaError_t allow_smem(F* f, size_t bytes) {
  return cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int NU>
gs_status launch_fwd(const gs_projected* proj, const gs_sorted* sorted, int n_pad, gs_frame fr, float* image,
                     float* final_T, uint32_t* n_contrib, float* image_tan, int32_t* status, cudaStream_t st) {
  const TileGrid g = tile_grid(fr);
  const int nthr = fr.tile_w * fr.tile_h / kPixPerThread, batch = fwd_batch(fr, nthr);
  const size_t smem = 16 + (size_t)batch * (2 * sizeof(Rec) * (1 + NU) + sizeof(uint32_t));
  // the dynamic shared-memory limit, raised as far as a launch needs
  const bool cb = fr.batch != 0, big = blend_threads(nthr) == 256;
  auto* kern = big ? (cb ? raster_fwd_kernel<NU, true, 256> : raster_fwd_kernel<NU, false, 256>)
                   : (cb ? raster_fwd_kernel<NU, true, 128> : raster_fwd_kernel<NU, false, 128>);
  static size_t attr[2][2] = {{0, 0}, {0, 0}};
  if (smem > attr[big][cb]) {
    if (allow_smem(kern, smem) != cudaSuccess) return check_launch("gs_raster_fwd: smem attribute");
    attr[big][cb] = smem;
  }
  const unsigned blocks = (unsigned)((size_t)fr.n_views * g.T);
  kern<<<blocks, nthr, smem, st>>>(reinterpret_cast<const float4*>(proj->rec),
                                   reinterpret_cast<const float4*>(proj->tangent), sorted->vals, sorted->ranges,
                                   sorted->order, n_pad,
                                   fr, g.Tx, g.T, image, final_T, n_contrib, image_tan, sorted->masks, status);
  return check_launch("gs_raster_fwd");
}

size_t bwd_cot_floats(int32_t n_pad, gs_frame fr, int streams) {
  return (size_t)fr.n_views * n_pad * cot_stride(streams);
}

// The reverse call's workspace: its header, the rows, and how many floats of
// them this call uses.
struct CotWs {
  CotHeader* hdr;
  float* cot;
  uint64_t floats;
};

// Point ws at the workspace and have the rows zero before the blend: the
// prepare kernel clears them unless the header says they already are.
cudaError_t cot_prepare(void* workspace, uint64_t floats, CotWs& ws, cudaStream_t st) {
  ws.hdr = reinterpret_cast<CotHeader*>(workspace);
  ws.cot = reinterpret_cast<float*>(reinterpret_cast<char*>(workspace) + kCotHeaderBytes);
  ws.floats = floats;
  const size_t n4 = floats / 4;  // rows are whole float4s
  const unsigned blocks = (unsigned)std::max<size_t>(1, std::min<size_t>((n4 + 255) / 256, 152 * 8));
  cot_prepare_kernel<<<blocks, 256, 0, st>>>(ws.hdr, reinterpret_cast<float4*>(ws.cot), n4);
  return cudaGetLastError();
}

template <int DEG, int NU, bool GRAD>
void launch_pbwd(const gs_params* x, const gs_camera* cams, gs_frame fr, CotWs ws, const gs_probe* probe,
                 float* grad, float* hz, cudaStream_t st) {
  constexpr int S = (GRAD ? 1 : 0) + NU;
  const size_t smem = pbwd_stash_bytes(fr.n_views, S);
  static size_t attr = 0;
  if (smem > attr) {
    if (allow_smem(project_bwd_kernel<DEG, NU, GRAD>, smem) != cudaSuccess) return;  // the caller reports the error
    attr = smem;
  }
  const dim3 pg((x->n + kPbwdThreads - 1) / kPbwdThreads), pb(kPbwdThreads);
  project_bwd_kernel<DEG, NU, GRAD><<<pg, pb, smem, st>>>(x->data, x->n, x->n_pad, cams, fr, ws.cot,
                                                          probe_arg(probe), grad, hz, ws.hdr, ws.floats);
}

// The reverse blend over the frame, then the projection's reverse pass: of the
// one scene x (ba NULL), or of each batch item from its slot (ba given: records
// and cotangents at pitch n_pad, each view its own objective, m = 3 H W).
template <int NU, bool GRAD>
void launch_bwd_kernels(const gs_params* x, const BatchArg* ba, int n_pad, int deg, const gs_camera* cams,
                        const gs_projected* proj, const gs_sorted* sorted, gs_frame fr, const float* image,
                        const float* target, const float* final_T, const uint32_t* n_contrib, const float* image_tan,
                        const gs_probe* probe, gs_loss loss, float* grad, float* hz, float* loss_out, CotWs ws,
                        int32_t* status, cudaStream_t st) {
  const TileGrid g = tile_grid(fr);
  const int nthr = fr.tile_w * fr.tile_h / kPixPerThread, batch = bwd_batch(fr, nthr);
  const size_t smem = bwd_smem_bytes(batch);
  const bool cb = fr.batch != 0, big = blend_threads(nthr) == 256;
  auto* kern = big ? (cb ? raster_bwd_kernel<NU, GRAD, true, 256> : raster_bwd_kernel<NU, GRAD, false, 256>)
                   : (cb ? raster_bwd_kernel<NU, GRAD, true, 128> : raster_bwd_kernel<NU, GRAD, false, 128>);
  static size_t attr[2][2] = {{0, 0}, {0, 0}};
  if (smem > 48 * 1024 && smem > attr[big][cb]) {
    if (allow_smem(kern, smem) != cudaSuccess) return;  // the caller reports the error
    attr[big][cb] = smem;
  }
  const double views_per_objective = ba ? 1.0 : (double)fr.n_views;
  const float inv_m = (float)(1.0 / (3.0 * (double)fr.width * fr.height * views_per_objective));
  const unsigned blocks = (unsigned)((size_t)fr.n_views * g.T);
  kern<<<blocks, nthr, smem, st>>>(
      reinterpret_cast<const float4*>(proj->rec), sorted->vals, sorted->ranges, sorted->order, n_pad, fr, g.Tx,
      g.T, image,
      target, final_T, n_contrib, image_tan, loss.kind, loss.gn_floor, inv_m, ws.cot, loss_out, ba ? 1 : 0, ws.hdr,
      sorted->masks, status);
  if (ba) {
    if (ba->first_block[ba->n_items] == 0) return;
    constexpr int S = (GRAD ? 1 : 0) + NU;
    const size_t sm = pbwd_stash_bytes(1, S);
    const ProbeArg pa = probe_arg(probe);
    const dim3 grid(ba->first_block[ba->n_items]), blk(kPbwdThreads);
#define GS_PBWD_BATCH(D)                                                                           \
  do {                                                                                             \
    static size_t battr = 0;                                                                       \
    if (sm > battr) {                                                                              \
      if (allow_smem(project_bwd_batch_kernel<D, NU, GRAD>, sm) != cudaSuccess) return;            \
      battr = sm;                                                                                  \
    }                                                                                              \
    project_bwd_batch_kernel<D, NU, GRAD><<<grid, blk, sm, st>>>(*ba, fr, ws.cot, n_pad, pa, ws.hdr, \
                                                                 ws.floats);                       \
  } while (0)
    switch (deg) {
      case 0: GS_PBWD_BATCH(0); break;
      case 1: GS_PBWD_BATCH(1); break;
      case 2: GS_PBWD_BATCH(2); break;
      default: GS_PBWD_BATCH(3); break;
    }
#undef GS_PBWD_BATCH
    return;
  }
  if (x->n == 0) return;
  switch (x->sh_degree) {
    case 0: launch_pbwd<0, NU, GRAD>(x, cams, fr, ws, probe, grad, hz, st); break;
    case 1: launch_pbwd<1, NU, GRAD>(x, cams, fr, ws, probe, grad, hz, st); break;
    case 2: launch_pbwd<2, NU, GRAD>(x, cams, fr, ws, probe, grad, hz, st); break;
    default: launch_pbwd<3, NU, GRAD>(x, cams, fr, ws, probe, grad, hz, st); break;
  }
}

// The kernels of one reverse call for the stream counts: the gradient stream
// (want_grad) and nu probe streams.
void launch_bwd_streams(bool want_grad, int nu, const gs_params* x, const BatchArg* ba, int n_pad, int deg,
                        const gs_camera* cams, const gs_projected* proj, const gs_sorted* sorted, gs_frame frame,
                        const float* image, const float* target, const float* final_T, const uint32_t* n_contrib,
                        const float* image_tangent, const gs_probe* probe, gs_loss loss, float* gptr, float* hptr,
                        float* loss_out, CotWs ws, int32_t* status, cudaStream_t st) {
#define GS_BWD_ARGS x, ba, n_pad, deg, cams, proj, sorted, frame, image, target, final_T, n_contrib, image_tangent, \
                    probe, loss, gptr, hptr, loss_out, ws, status, st
  if (want_grad) {
    if (nu == 0) launch_bwd_kernels<0, true>(GS_BWD_ARGS);
    else if (nu == 1) launch_bwd_kernels<1, true>(GS_BWD_ARGS);
    else launch_bwd_kernels<2, true>(GS_BWD_ARGS);
  } else {
    if (nu == 1) launch_bwd_kernels<1, false>(GS_BWD_ARGS);
    else launch_bwd_kernels<2, false>(GS_BWD_ARGS);
  }
#undef GS_BWD_ARGS
}

gs_status run_bwd(bool want_grad, const gs_params* x, const gs_camera* cams, gs_frame frame, const gs_projected* proj,
                  const gs_sorted* sorted, const float* image, const float* target, const float* final_T,
                  const uint32_t* n_contrib, const float* image_tangent, const gs_probe* probe, gs_loss loss,
                  gs_params* grad, gs_params* hz, float* loss_out, void* workspace, size_t workspace_bytes,
                  int32_t* status, void* stream, const char* name) {
  GS_REQUIRE(x && cams && proj && sorted && image && target && final_T && n_contrib, "%s: null argument", name);
  GS_REQUIRE(proj->rec && sorted->vals && sorted->ranges && x->data, "%s: null device buffer", name);
  GS_REQUIRE(frame_ok(frame), "%s: bad frame", name);
  GS_REQUIRE(x->n >= 0 && x->n_pad >= x->n && x->n_pad % 4 == 0, "%s: bad n/n_pad", name);
  GS_REQUIRE(loss.kind == GS_LOSS_L1 || loss.kind == GS_LOSS_L2 || loss.kind == GS_LOSS_COTANGENT ||
                 loss.kind == GS_LOSS_WEIGHTED,
             "%s: bad loss kind %d", name, loss.kind);
  const bool given = loss.kind == GS_LOSS_COTANGENT;
  const int nu = ((image_tangent || given) && probe) ? probe->nu : 0;
  GS_REQUIRE(loss.kind != GS_LOSS_WEIGHTED || nu == 0 || image_tangent, "%s: weighted loss needs image_tangent",
             name);
  if (nu < 0 || nu > 2 || x->sh_degree < 0 || x->sh_degree > 3) {
    set_error("%s: unsupported nu=%d sh_degree=%d", name, nu, x->sh_degree);
    return GS_ERR_UNSUPPORTED;
  }
  GS_REQUIRE(want_grad || nu > 0, "%s: needs image_tangent and a probe with nu >= 1", name);
  GS_REQUIRE(!want_grad || (grad && grad->data), "%s: null grad", name);
  GS_REQUIRE(nu == 0 || (hz && hz->data), "%s: probes given but hz is NULL", name);
  auto same = [&](const gs_params* p) { return !p || (p->n == x->n && p->n_pad == x->n_pad && p->sh_degree == x->sh_degree); };
  GS_REQUIRE(same(grad) && same(hz), "%s: grad/hz layout differs from x", name);
  const int streams = (want_grad ? 1 : 0) + nu;
  const size_t floats = bwd_cot_floats(x->n_pad, frame, streams);
  const size_t need = kCotHeaderBytes + floats * sizeof(float);
  GS_REQUIRE(workspace && workspace_bytes >= need, "%s: workspace needs %zu bytes, got %zu", name, need,
             workspace_bytes);
  GS_REQUIRE(((uintptr_t)workspace & 15) == 0, "%s: workspace must be 16-byte aligned", name);
  cudaStream_t st = (cudaStream_t)stream;
  CotWs ws;
  if (cot_prepare(workspace, floats, ws, st) != cudaSuccess) return check_launch(name);
  float* gptr = want_grad ? grad->data : nullptr;
  float* hptr = nu ? hz->data : nullptr;
  launch_bwd_streams(want_grad, nu, x, nullptr, x->n_pad, x->sh_degree, cams, proj, sorted, frame, image, target,
                     final_T, n_contrib, image_tangent, probe, loss, gptr, hptr, loss_out, ws, status, st);
  return check_launch(name);
}

}  // namespace
}  // namespace gs

extern "C" gs_status gs_raster_fwd(const gs_projected* proj, const gs_sorted* sorted, int32_t n_pad, gs_frame frame,
                                   const gs_probe* probe, float* image, float* final_T, uint32_t* n_contrib,
                                   float* image_tangent, int32_t* status, void* stream) {
  using namespace gs;
  GS_REQUIRE(proj && sorted && proj->rec && sorted->vals && sorted->ranges, "gs_raster_fwd: null argument");
  GS_REQUIRE(image && final_T && n_contrib, "gs_raster_fwd: null output");
  GS_REQUIRE(frame_ok(frame), "gs_raster_fwd: bad frame (tile %dx%d)", frame.tile_w, frame.tile_h);
  GS_REQUIRE(n_pad >= 0 && n_pad % 4 == 0, "gs_raster_fwd: bad n_pad");
  const int nu = (probe && image_tangent) ? probe->nu : 0;
  if (nu < 0 || nu > 2) {
    set_error("gs_raster_fwd: unsupported nu=%d", nu);
    return GS_ERR_UNSUPPORTED;
  }
  GS_REQUIRE(nu == 0 || proj->tangent, "gs_raster_fwd: probes given but proj->tangent is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  if (nu == 0) return launch_fwd<0>(proj, sorted, n_pad, frame, image, final_T, n_contrib, nullptr, status, st);
  if (nu == 1) return launch_fwd<1>(proj, sorted, n_pad, frame, image, final_T, n_contrib, image_tangent, status, st);
  return launch_fwd<2>(proj, sorted, n_pad, frame, image, final_T, n_contrib, image_tangent, status, st);
}

extern "C" size_t gs_raster_bwd_workspace_size(int32_t n_pad, gs_frame frame, int32_t nu) {
  if (n_pad < 0 || nu < 0 || nu > 2 || !gs::frame_ok(frame)) return 0;
  return gs::kCotHeaderBytes + gs::bwd_cot_floats(n_pad, frame, 1 + nu) * sizeof(float);
}

extern "C" gs_status gs_raster_bwd(const gs_params* x, const gs_camera* cams, gs_frame frame, const gs_projected* proj,
                                   const gs_sorted* sorted, const float* image, const float* target,
                                   const float* final_T, const uint32_t* n_contrib, const float* image_tangent,
                                   const gs_probe* probe, gs_loss loss, gs_params* grad, gs_params* hz,
                                   float* loss_out, void* workspace, size_t workspace_bytes, int32_t* status,
                                   void* stream) {
  return gs::run_bwd(true, x, cams, frame, proj, sorted, image, target, final_T, n_contrib, image_tangent, probe, loss,
                     grad, hz, loss_out, workspace, workspace_bytes, status, stream, "gs_raster_bwd");
}

extern "C" gs_status gs_hvp_diag(const gs_params* x, const gs_camera* cams, gs_frame frame, const gs_projected* proj,
                                 const gs_sorted* sorted, const float* image, const float* target, const float* final_T,
                                 const uint32_t* n_contrib, const float* image_tangent, const gs_probe* probe,
                                 gs_loss loss, gs_params* hz, void* workspace, size_t workspace_bytes, int32_t* status,
                                 void* stream) {
  return gs::run_bwd(false, x, cams, frame, proj, sorted, image, target, final_T, n_contrib, image_tangent, probe, loss,
                     nullptr, hz, nullptr, workspace, workspace_bytes, status, stream, "gs_hvp_diag");
}

extern "C" gs_status gs_raster_bwd_batch(const gs_batch_item* items, int32_t n_items, int32_t n_pad_max,
                                         gs_frame frame, const gs_projected* proj, const gs_sorted* sorted,
                                         const float* image, const float* target, const float* final_T,
                                         const uint32_t* n_contrib, const float* image_tangent, const gs_probe* probe,
                                         gs_loss loss, float* loss_out, void* workspace, size_t workspace_bytes,
                                         int32_t* status, void* stream) {
  using namespace gs;
  const char* name = "gs_raster_bwd_batch";
  GS_REQUIRE(items && proj && sorted && image && target && final_T && n_contrib, "%s: null argument", name);
  GS_REQUIRE(proj->rec && sorted->vals && sorted->ranges, "%s: null device buffer", name);
  GS_REQUIRE(n_items >= 1 && n_items <= GS_BATCH_MAX, "%s: n_items=%d outside [1, %d]", name, n_items, GS_BATCH_MAX);
  GS_REQUIRE(frame_ok(frame) && frame.n_views == n_items, "%s: bad frame (n_views must equal n_items)", name);
  GS_REQUIRE(n_pad_max >= 4 && n_pad_max % 4 == 0, "%s: bad n_pad_max=%d", name, n_pad_max);
  GS_REQUIRE(loss.kind == GS_LOSS_L1 || loss.kind == GS_LOSS_L2 || loss.kind == GS_LOSS_COTANGENT ||
                 loss.kind == GS_LOSS_WEIGHTED,
             "%s: bad loss kind %d", name, loss.kind);
  const bool given = loss.kind == GS_LOSS_COTANGENT;
  const int nu = ((image_tangent || given) && probe) ? probe->nu : 0;
  const int deg = items[0].x.sh_degree;
  if (nu < 0 || nu > 2 || deg < 0 || deg > 3) {
    set_error("%s: unsupported nu=%d sh_degree=%d", name, nu, deg);
    return GS_ERR_UNSUPPORTED;
  }
  GS_REQUIRE(loss.kind != GS_LOSS_WEIGHTED || nu == 0 || image_tangent, "%s: weighted loss needs image_tangent",
             name);
  for (int b = 0; b < n_items; ++b) {
    const gs_batch_item& it = items[b];
    auto same = [&](const gs_params& p) { return p.n == it.x.n && p.n_pad == it.x.n_pad && p.sh_degree == deg; };
    GS_REQUIRE(it.x.data && it.cam && it.grad.data && same(it.x) && same(it.grad),
               "%s: item %d needs x, cam and a gradient of x's layout", name, b);
    GS_REQUIRE(nu == 0 || (it.hz.data && same(it.hz) && it.t >= 1), "%s: item %d needs hz and t >= 1 with probes",
               name, b);
    GS_REQUIRE(it.x.n >= 0 && it.x.n <= n_pad_max && it.x.n_pad % 4 == 0, "%s: item %d: bad n=%d n_pad=%d", name,
               b, it.x.n, it.x.n_pad);
  }
  const size_t floats = bwd_cot_floats(n_pad_max, frame, 1 + nu);
  const size_t need = kCotHeaderBytes + floats * sizeof(float);
  GS_REQUIRE(workspace && workspace_bytes >= need, "%s: workspace needs %zu bytes, got %zu", name, need,
             workspace_bytes);
  GS_REQUIRE(((uintptr_t)workspace & 15) == 0, "%s: workspace must be 16-byte aligned", name);
  cudaStream_t st = (cudaStream_t)stream;
  CotWs ws;
  if (cot_prepare(workspace, floats, ws, st) != cudaSuccess) return check_launch(name);
  const BatchArg ba = batch_arg(items, n_items, [](const gs_batch_item& it) {
    return (it.x.n + kPbwdThreads - 1) / kPbwdThreads;
  });
  launch_bwd_streams(true, nu, nullptr, &ba, n_pad_max, deg, nullptr, proj, sorted, frame, image, target, final_T,
                     n_contrib, image_tangent, probe, loss, nullptr, nullptr, loss_out, ws, status, st);
  return check_launch(name);
}
