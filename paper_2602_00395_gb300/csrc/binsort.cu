// gs_bin_sort: tile binning and depth order of the tile-based rasteriser
// (Sec. 3.1 of arXiv 2602.00395).
//
// Every pair of one splat shares its depth, so the order (tile, depth, splat)
// is built in two stages instead of sorting 64-bit (tile, depth) pair keys:
//
//   records  per (view, splat): its tiles (the FP32 rectangle, narrowed row
//            by row to the footprint ellipse, see row_span_v); the V x n_pad
//            records are sorted by (view, depth bits) with a stable LSD radix
//            sort (record index order breaks ties)
//   scan     emission offsets in that order and the pair count P
//   emit     key = view * tiles + tile (32 bits), value = splat, written in
//            (view, depth, splat) order
//   sort     stable LSD radix sort of the pairs on those keys: the depth order
//            within a tile is the emission order, so no depth bits are moved
//   ranges   [start, end) of every tile
//
// Each radix pass is a per-block digit histogram, a device-wide scan of the
// histograms, and a scatter that ranks each block's keys stably in shared
// memory and writes every digit's run contiguously; no block waits on another.
// The result is the total order (key, splat index).  Grids are sized by the
// pair capacity and read P from device memory, so the call needs no host
// synchronisation (and can be captured in a graph).
#include "common.cuh"

namespace gs {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanChunk = kScanThreads * kScanItems;  // 2048
// Items per thread of a radix tile, and the scatter's resident blocks per SM
// (its launch bound); overridable at build time for sweeps.
#ifndef GS_RADIX_ITEMS
#define GS_RADIX_ITEMS 8
#endif
#ifndef GS_RADIX_MIN_BLOCKS
#define GS_RADIX_MIN_BLOCKS 4
#endif
constexpr int kRadixThreads = 256;
constexpr int kRadixItems = GS_RADIX_ITEMS;
constexpr int kRadixTile = kRadixThreads * kRadixItems;  // 2048 by default
constexpr int kRadixWarps = kRadixThreads / 32;

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// The tile rows of record g (see foot_rows).
__device__ __forceinline__ FootRows record_rows(const float4* __restrict__ rec, size_t g, const gs_frame& fr, int Tx,
                                                int Ty, float& depth) {
  const float4 a = rec[3 * g + 0];
  const float4 b = rec[3 * g + 1];
  const float4 c = rec[3 * g + 2];
  depth = c.y;
  const int r = __float_as_int(c.z);
  FootRows f = foot_rows(a.x, a.y, a.z, a.w, b.x, r, __float_as_uint(c.w), fr.footprint_bins != 0, fr.tile_w,
                         fr.tile_h, Tx, Ty);
  if (r <= 0) f.x1 = f.x0;  // culled: no tiles
  return f;
}

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t& total, uint32_t* s_warp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    uint32_t w = lane < nw ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) s_warp[lane] = w;
  }
  __syncthreads();
  total = s_warp[(blockDim.x >> 5) - 1];
  const uint32_t before = warp > 0 ? s_warp[warp - 1] : 0;
  __syncthreads();
  return before + x - v;
}

// ------------------------------------------------------------------ records
// Per record g: counts[g] = its pairs; rkeys[g] = bits(depth) (then sorted
// within each view's segment); rvals[g] = g; and its row table for the emit:
// one entry per row of its rectangle, (pairs in the rows above, first tile),
// allocated from `rows` by one atomic per block, and the header
// hdr[g] = (bits(depth), first row | rows << 16, table offset, pairs).  The
// table holds at most 2 empty rows per record beyond its pairs (non-empty rows
// are contiguous), so rows_cap = pair capacity + 2 x records overflows only with
// the pairs; then the record keeps no table and GS_FLAG_CAPACITY is raised.
__global__ void record_keys_kernel(const float4* __restrict__ rec, int n_pad, gs_frame fr, int Tx, int Ty,
                                   uint32_t* __restrict__ counts, uint32_t* __restrict__ rkeys,
                                   uint32_t* __restrict__ rvals, uint4* __restrict__ hdr, uint2* __restrict__ rows,
                                   uint64_t rows_cap, uint32_t* __restrict__ rows_used, int32_t* __restrict__ status) {
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_base;
  const size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = g < (size_t)fr.n_views * n_pad;
  float depth = 0.f;
  FootRows f{};
  uint32_t R = 0;
  if (in) {
    f = record_rows(rec, g, fr, Tx, Ty, depth);
    if (f.x1 > f.x0 && f.y1 > f.y0) R = (uint32_t)(f.y1 - f.y0);
  }
  uint32_t total;
  const uint32_t ex = block_exclusive_scan(R, total, s_warp);
  if (threadIdx.x == 0) s_base = total ? atomicAdd(rows_used, total) : 0u;
  __syncthreads();
  if (!in) return;
  const uint32_t off = s_base + ex;
  uint32_t cnt = 0;
  if (R && (uint64_t)off + R <= rows_cap) {
    float vlo = f.exact ? band_v(f, f.y0 * fr.tile_h) : 0.f;
    for (uint32_t k = 0; k < R; ++k) {
      int a, b;
      if (f.exact) {
        const float vhi = band_v(f, (f.y0 + (int)k + 1) * fr.tile_h);
        row_span_v(f, vlo, vhi, fr.tile_w, Tx, a, b);
        vlo = vhi;
      } else {
        a = f.x0;
        b = f.x1;
      }
      rows[(size_t)off + k] = make_uint2(cnt, (uint32_t)a);
      cnt += (uint32_t)(b - a);
    }
  } else if (R) {
    cnt = foot_count(f, fr.tile_w, fr.tile_h, Tx);
    R = 0;
    if (status) atomicOr(status, GS_FLAG_CAPACITY);
  }
  counts[g] = cnt;
  hdr[g] = make_uint4(__float_as_uint(depth), (uint32_t)f.y0 | (R << 16), off, cnt);
  rkeys[g] = __float_as_uint(depth);
  rvals[g] = (uint32_t)g;
}

// scnt[p] = counts of the record at sorted position p
__global__ void gather_counts_kernel(const uint32_t* __restrict__ order, const uint32_t* __restrict__ counts,
                                     uint32_t* __restrict__ scnt, size_t items) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < items) scnt[p] = counts[order[p]];
}

// ------------------------------------------------------------------- scan
// Length of a scan: n, or, when `pairs` is given, the radix histogram length
// 256 * ceil(min(*pairs, capacity) / tile) of the pairs in use.
__device__ __forceinline__ size_t scan_length(size_t n, const uint32_t* pairs, uint64_t capacity) {
  if (!pairs) return n;
  const uint64_t p = *pairs < capacity ? *pairs : capacity;
  return (size_t)256 * (size_t)((p + kRadixTile - 1) / kRadixTile);
}

__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const uint32_t* __restrict__ in, size_t n_host,
                                                                   const uint32_t* pairs, uint64_t capacity,
                                                                   uint32_t* __restrict__ block_sums) {
  __shared__ uint32_t s_warp[32];
  const size_t n = scan_length(n_host, pairs, capacity);
  const size_t base = (size_t)blockIdx.x * kScanChunk;
  if (base >= n) return;
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    size_t idx = base + (size_t)k * kScanThreads + threadIdx.x;
    if (idx < n) s += in[idx];
  }
  uint32_t total;
  block_exclusive_scan(s, total, s_warp);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// One block: exclusive scan of the block sums; the grand total goes to *total
// (and, if capacity is non-zero, GS_FLAG_CAPACITY is raised when it exceeds it).
__global__ void __launch_bounds__(1024) scan_blocks_kernel(uint32_t* __restrict__ sums, size_t n_host,
                                                           const uint32_t* pairs, uint64_t pair_capacity,
                                                           uint32_t* __restrict__ total, uint64_t capacity,
                                                           int32_t* __restrict__ status) {
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_carry;
  const int nb = (int)((scan_length(n_host, pairs, pair_capacity) + kScanChunk - 1) / kScanChunk);
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += blockDim.x) {
    const int idx = base + threadIdx.x;
    const uint32_t v = idx < nb ? sums[idx] : 0;
    uint32_t chunk_total;
    const uint32_t ex = block_exclusive_scan(v, chunk_total, s_warp);
    const uint32_t carry = s_carry;
    if (idx < nb) sums[idx] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) s_carry = carry + chunk_total;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (total) *total = s_carry;
    if (capacity && (uint64_t)s_carry > capacity && status) atomicOr(status, GS_FLAG_CAPACITY);
  }
}

__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const uint32_t* in, uint32_t* out, size_t n_host,
                                                                  const uint32_t* pairs, uint64_t capacity,
                                                                  const uint32_t* __restrict__ block_sums) {
  __shared__ uint32_t s_warp[32];
  const size_t n = scan_length(n_host, pairs, capacity);
  if ((size_t)blockIdx.x * kScanChunk >= n) return;
  const size_t base = (size_t)blockIdx.x * kScanChunk + (size_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0u;
    s += v[k];
  }
  uint32_t total;
  uint32_t run = block_exclusive_scan(s, total, s_warp) + block_sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
}

// The whole scan in one block of 1024 threads (chunks of 8192 entries with a
// carried total), for lengths where three dependent launches would cost more
// than the work: the short histograms of small scenes.
constexpr size_t kSingleScanMax = 65536;
__global__ void __launch_bounds__(1024) scan_single_kernel(const uint32_t* in, uint32_t* out, size_t n_host,
                                                           const uint32_t* pairs, uint64_t pair_capacity,
                                                           uint32_t* __restrict__ total, uint64_t capacity,
                                                           int32_t* __restrict__ status) {
  __shared__ uint32_t s_warp[32];
  const size_t n = scan_length(n_host, pairs, pair_capacity);
  uint32_t carry = 0;
  for (size_t base = 0; base < n; base += (size_t)1024 * kScanItems) {
    const size_t b = base + (size_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      v[k] = b + k < n ? in[b + k] : 0u;
      s += v[k];
    }
    uint32_t tot;
    uint32_t run = block_exclusive_scan(s, tot, s_warp) + carry;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      if (b + k < n) out[b + k] = run;
      run += v[k];
    }
    carry += tot;
  }
  if (threadIdx.x == 0) {
    if (total) *total = carry;
    if (capacity && (uint64_t)carry > capacity && status) atomicOr(status, GS_FLAG_CAPACITY);
  }
}

inline int scan_blocks(size_t n) { return (int)((n + kScanChunk - 1) / kScanChunk); }

// in -> out exclusive scan of n_max entries (in may equal out).  If `pairs` is
// given, only the radix histogram of the pairs in use is scanned (n_max bounds
// it).  The grand total goes to *total; GS_FLAG_CAPACITY is raised when it
// exceeds a non-zero `capacity`.
void exclusive_scan(const uint32_t* in, uint32_t* out, size_t n_max, const uint32_t* pairs, uint64_t pair_capacity,
                    uint32_t* block_sums, uint32_t* total, uint64_t capacity, int32_t* status, cudaStream_t st) {
  const int nb = scan_blocks(n_max);
  if (nb == 0) return;
  if (n_max <= kSingleScanMax) {
    scan_single_kernel<<<1, 1024, 0, st>>>(in, out, n_max, pairs, pair_capacity, total, capacity, status);
    return;
  }
  scan_reduce_kernel<<<nb, kScanThreads, 0, st>>>(in, n_max, pairs, pair_capacity, block_sums);
  scan_blocks_kernel<<<1, 1024, 0, st>>>(block_sums, n_max, pairs, pair_capacity, total, capacity, status);
  scan_apply_kernel<<<nb, kScanThreads, 0, st>>>(in, out, n_max, pairs, pair_capacity, block_sums);
}

// ------------------------------------------------------------------- emit
// One warp emits the pairs of 32 consecutive records in (view, depth) order.
// Their output ranges are contiguous (the offsets are an exclusive scan in that
// order), so the warp writes its whole range with consecutive lanes on
// consecutive pairs; each lane finds the record that owns its pair by a binary
// search over the warp's prefix sums, and the pair's row by a binary search
// over that record's row table (see record_keys_kernel).
__global__ void emit_kernel(const uint4* __restrict__ hdr, const uint2* __restrict__ rows, int n_pad, gs_frame fr,
                            int Tx, int Ty, const uint32_t* __restrict__ order, const uint32_t* __restrict__ offsets,
                            uint64_t capacity, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const size_t G = (size_t)fr.n_views * n_pad;
  const size_t p0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // sorted record position
  const size_t w0 = p0 - (threadIdx.x & 31);
  if (w0 >= G) return;  // whole warp
  const int lane = threadIdx.x & 31;
  uint32_t g = 0;
  uint4 h = make_uint4(0u, 0u, 0u, 0u);
  if (p0 < G) {
    g = order[p0];
    h = hdr[g];
  }
  // this lane's record as (first tile key of its view, splat index): one
  // division per record instead of one per pair (views x tiles < 2^32)
  const uint32_t gview = g / (uint32_t)n_pad;
  const uint32_t gkey0 = gview * (uint32_t)(Tx * Ty), gsplat = g - gview * (uint32_t)n_pad;
  const uint32_t cnt = h.w;
  // inclusive warp scan of the counts
  uint32_t incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const uint32_t start = incl - cnt;
  const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
  const uint64_t base = offsets[w0];
  const uint32_t rounds = (total + 31) / 32;
  for (uint32_t rd = 0; rd < rounds; ++rd) {
    const uint32_t p = rd * 32 + lane;
    // owner = largest lane whose start <= p (lanes with no pairs never win over the next lane)
    int lo = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
      const int cand = lo + step;
      const uint32_t sc = __shfl_sync(0xffffffffu, start, cand & 31);
      if (cand < 32 && sc <= p) lo = cand;
    }
    const uint32_t o_start = __shfl_sync(0xffffffffu, start, lo);
    const uint32_t okey0 = __shfl_sync(0xffffffffu, gkey0, lo);
    const uint32_t osplat = __shfl_sync(0xffffffffu, gsplat, lo);
    const uint32_t oyr = __shfl_sync(0xffffffffu, h.y, lo);
    const uint32_t ooff = __shfl_sync(0xffffffffu, h.z, lo);
    const uint32_t R = oyr >> 16;
    const uint64_t at = base + p;
    if (p < total && at < capacity) {
      uint32_t tile = okey0;
      if (R > 0) {
        const uint32_t q = p - o_start;
        // last row whose pairs above are <= q (empty rows repeat the count before them)
        uint32_t a = 0, b = R - 1;
        while (a < b) {
          const uint32_t mid = (a + b + 1) >> 1;
          if (__ldg(&rows[(size_t)ooff + mid].x) <= q) a = mid; else b = mid - 1;
        }
        const uint2 e = __ldg(&rows[(size_t)ooff + a]);
        // q - e.x < the row's pairs, so txx stays in the row; the clamp only
        // keeps every tile index inside the view if that ever failed
        const uint32_t txx = min(e.y + (q - e.x), (uint32_t)(Tx - 1));
        tile += ((oyr & 0xffffu) + a) * (uint32_t)Tx + txx;
      }
      // (R == 0 with pairs: the record's row table did not fit, which happens
      // only when the pairs exceed the capacity and GS_FLAG_CAPACITY is raised;
      // its slots still get a valid tile and splat so that every slot below the
      // capacity holds an in-range pair)
      keys[at] = tile;
      vals[at] = osplat;
    }
  }
}

// ------------------------------------------------------------ radix passes
// A pass sorts nseg segments independently and stably on one 8-bit digit.
// Segment g holds items [g * stride, g * stride + len): the record sort has one
// segment per view (len = stride = n_pad), the pair sort one segment whose
// length is the pair count P in device memory.  Each segment is cut into
// tiles of kRadixTile items, tile t of segment g handled by block g * bpg + t
// (blocks past the segment's tiles return).  The digit histograms are stored
// segment-major, then digit, then tile: hist[(g * 256 + d) * bps + t], so that
// one exclusive scan of all of them gives every (segment, digit, tile) its
// first output position.
struct Seg {
  const uint32_t* len_dev;  // device length of the single segment, or null
  uint64_t cap;             // clamp of *len_dev
  uint32_t len;             // host length of every segment (len_dev == null)
  uint32_t stride;          // items between segment starts
};

__device__ __forceinline__ uint32_t seg_len(const Seg& sg) {
  if (!sg.len_dev) return sg.len;
  const uint64_t p = *sg.len_dev;
  return (uint32_t)(p < sg.cap ? p : sg.cap);
}

template <typename K>
__device__ __forceinline__ uint32_t digit_of(K key, int shift) {
  return (uint32_t)(key >> shift) & 255u;
}

// Digit counts of one tile.  A thread counts kRadixItems consecutive keys (read
// as 16-byte vectors) and adds each run of equal digits to the block's
// counters with one shared atomic: a splat's pairs are adjacent and share their
// high tile digit, so runs are common.
template <typename K>
__device__ __forceinline__ void load_run(const K* p, K (&kk)[kRadixItems]) {
  static_assert((kRadixItems * sizeof(K)) % 16 == 0, "vector loads");
  const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
  for (int v = 0; v < (int)(kRadixItems * sizeof(K) / 16); ++v) {
    const uint4 w = __ldg(q + v);
    memcpy(reinterpret_cast<char*>(kk) + 16 * v, &w, 16);
  }
}

template <typename K>
__global__ void __launch_bounds__(kRadixThreads) radix_hist_kernel(const K* __restrict__ keys, Seg sg, int bpg,
                                                                   int shift, uint32_t* __restrict__ hist) {
  __shared__ uint32_t s_cnt[256];
  const uint32_t len = seg_len(sg);
  const int g = blockIdx.x / bpg, t = blockIdx.x - g * bpg;
  const uint32_t bps = (len + kRadixTile - 1) / kRadixTile;
  if ((uint32_t)t >= bps) return;
  s_cnt[threadIdx.x] = 0;
  __syncthreads();
  const K* kin = keys + (size_t)g * sg.stride;
  const uint32_t base = (uint32_t)t * kRadixTile + threadIdx.x * kRadixItems;
  K kk[kRadixItems];
  if (base + kRadixItems <= len) {
    load_run(kin + base, kk);
  } else {
#pragma unroll
    for (int k = 0; k < kRadixItems; ++k) kk[k] = base + k < len ? kin[base + k] : (K)0;
  }
  uint32_t prev = 256u, run = 0;
#pragma unroll
  for (int k = 0; k < kRadixItems; ++k) {
    const uint32_t d = base + k < len ? digit_of(kk[k], shift) : 256u;
    if (d != prev) {
      if (run) atomicAdd(&s_cnt[prev], run);
      prev = d;
      run = 0;
    }
    run += d < 256u;
  }
  if (run) atomicAdd(&s_cnt[prev], run);
  __syncthreads();
  hist[((size_t)g * 256 + threadIdx.x) * bps + t] = s_cnt[threadIdx.x];
}

// Stable scatter of one tile.  Warp w owns the tile's items
// [w * 32 * kRadixItems, (w + 1) * 32 * kRadixItems), item k of lane L at
// offset k * 32 + L, so the warps' strips and the items within a strip are in
// input order.  Each warp ranks its strip against private digit counters (one
// match per item, no block barrier); the per-digit prefix over the warps and
// the tile's digit starts follow from one block scan; the keys are reordered by
// (digit, rank) in shared memory and each digit's run written contiguously.
template <typename K>
__global__ void __launch_bounds__(kRadixThreads, GS_RADIX_MIN_BLOCKS) radix_scatter_kernel(const K* __restrict__ kin_all,
                                                                      const uint32_t* __restrict__ vin_all,
                                                                      K* __restrict__ kout, uint32_t* __restrict__ vout,
                                                                      Seg sg, int bpg, int shift,
                                                                      const uint32_t* __restrict__ hist_scanned) {
  __shared__ K s_keys[kRadixTile];
  __shared__ uint32_t s_vals[kRadixTile];
  __shared__ uint32_t s_wc[kRadixWarps][256];  // per-warp digit counts, then their prefix over warps
  __shared__ uint32_t s_start[256];           // first tile position of each digit
  __shared__ uint32_t s_gofs[256];            // output position minus tile position, per digit
  __shared__ uint32_t s_warp[32];
  const uint32_t len = seg_len(sg);
  const int g = blockIdx.x / bpg, t = blockIdx.x - g * bpg;
  const uint32_t bps = (len + kRadixTile - 1) / kRadixTile;
  if ((uint32_t)t >= bps) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lt = lanemask_lt();
  const K* kin = kin_all + (size_t)g * sg.stride;
  const uint32_t* vin = vin_all + (size_t)g * sg.stride;
  const uint32_t base = (uint32_t)t * kRadixTile + (uint32_t)warp * 32 * kRadixItems + lane;
  K key[kRadixItems];
  uint32_t vv[kRadixItems], rank[kRadixItems], dg[kRadixItems];
#pragma unroll
  for (int k = 0; k < kRadixItems; ++k) {
    const uint32_t idx = base + (uint32_t)k * 32;
    key[k] = idx < len ? kin[idx] : (K)0;
    vv[k] = idx < len ? vin[idx] : 0u;
  }
#pragma unroll
  for (int q = lane; q < 256; q += 32) s_wc[warp][q] = 0;
  __syncwarp();
#pragma unroll
  for (int k = 0; k < kRadixItems; ++k) {
    const bool ok = base + (uint32_t)k * 32 < len;
    const uint32_t d = ok ? digit_of(key[k], shift) : 256u;
    dg[k] = d;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t before = ok ? s_wc[warp][d] : 0u;
    rank[k] = before + (uint32_t)__popc(peers & lt);
    __syncwarp();
    if (ok && (peers & lt) == 0) s_wc[warp][d] = before + (uint32_t)__popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // digit tid: prefix of the warps' counts, the tile's count, its start
  uint32_t run = 0;
#pragma unroll
  for (int w = 0; w < kRadixWarps; ++w) {
    const uint32_t c = s_wc[w][tid];
    s_wc[w][tid] = run;
    run += c;
  }
  uint32_t tot;
  const uint32_t start = block_exclusive_scan(run, tot, s_warp);
  s_start[tid] = start;
  s_gofs[tid] = hist_scanned[((size_t)g * 256 + tid) * bps + t] - start;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kRadixItems; ++k) {
    if (dg[k] < 256u) {
      const uint32_t pos = s_start[dg[k]] + s_wc[warp][dg[k]] + rank[k];
      s_keys[pos] = key[k];
      s_vals[pos] = vv[k];
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kRadixItems; ++k) {
    const uint32_t p = (uint32_t)k * kRadixThreads + tid;
    if (p < tot) {
      const K kk = s_keys[p];
      const size_t at = (size_t)s_gofs[digit_of(kk, shift)] + p;
      kout[at] = kk;
      vout[at] = s_vals[p];
    }
  }
}

// ------------------------------------------------------------------ ranges
__device__ __forceinline__ uint32_t pairs_in_use(const uint32_t* n_pairs, uint64_t capacity) {
  const uint64_t p = *n_pairs;
  return (uint32_t)(p < capacity ? p : capacity);
}

// A thread looks at four consecutive keys (one 16-byte load) and the key after
// them; a tile starts where its key differs from the previous one and ends
// where it differs from the next.
__global__ void ranges_kernel(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ n_pairs,
                              uint64_t capacity, uint64_t n_tiles, uint32_t* __restrict__ ranges) {
  const uint32_t P = pairs_in_use(n_pairs, capacity);
  const size_t step = (size_t)gridDim.x * blockDim.x * 4;
  for (size_t p0 = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * 4; p0 < P; p0 += step) {
    uint32_t tl[5];
    if (p0 + 4 <= P) {
      const uint4 a = __ldg(reinterpret_cast<const uint4*>(keys + p0));
      tl[0] = a.x; tl[1] = a.y; tl[2] = a.z; tl[3] = a.w;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) tl[k] = p0 + k < P ? keys[p0 + k] : 0xffffffffu;
    }
    tl[4] = p0 + 4 < P ? keys[p0 + 4] : 0xffffffffu;
    uint32_t prev = p0 > 0 ? keys[p0 - 1] : 0xffffffffu;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const size_t p = p0 + k;
      if (p < P && tl[k] < n_tiles) {  // every emitted tile is below n_tiles; the test guards the writes
        if (tl[k] != prev) ranges[2 * (size_t)tl[k]] = (uint32_t)p;
        if (tl[k + 1] != tl[k]) ranges[2 * (size_t)tl[k] + 1] = (uint32_t)(p + 1);
      }
      prev = tl[k];
    }
  }
}

// ------------------------------------------------------------- tile order
// The blends run one block per tile; starting the longest lists first keeps a
// few heavy tiles from running alone at the end.  A tile's class is
// 8 * floor(log2 len) + the next 3 bits of len (256 classes, 0 for an empty
// list); the order is a counting sort by class, heaviest first.
__device__ __forceinline__ uint32_t tile_class(uint32_t len) {
  if (len == 0) return 0;
  const int e = 31 - __clz(len);
  const uint32_t m = e >= 3 ? (len >> (e - 3)) & 7u : (len << (3 - e)) & 7u;
  return min(255u, 1u + 8u * (uint32_t)e + m);
}

__global__ void tile_class_count_kernel(const uint32_t* __restrict__ ranges, uint32_t n_tiles,
                                        uint32_t* __restrict__ cls_count) {
  __shared__ uint32_t s_cnt[256];
  s_cnt[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n_tiles) atomicAdd(&s_cnt[tile_class(ranges[2 * t + 1] - ranges[2 * t])], 1u);
  __syncthreads();
  if (s_cnt[threadIdx.x]) atomicAdd(&cls_count[threadIdx.x], s_cnt[threadIdx.x]);
}

// cls_count -> the first slot of each class, heaviest class first (one block of 256)
__global__ void tile_class_starts_kernel(uint32_t* __restrict__ cls_count) {
  __shared__ uint32_t s_warp[32];
  const uint32_t c = cls_count[255 - threadIdx.x];  // thread k holds class 255 - k
  uint32_t total;
  const uint32_t ex = block_exclusive_scan(c, total, s_warp);
  cls_count[255 - threadIdx.x] = ex;
}

__global__ void tile_order_kernel(const uint32_t* __restrict__ ranges, uint32_t n_tiles,
                                  uint32_t* __restrict__ cls_next, uint32_t* __restrict__ order) {
  // one atomic per class present in the warp (most tiles share class 0, the
  // empty lists); a warp's tiles of one class keep their index order
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x, lane = threadIdx.x & 31;
  const uint32_t c = t < n_tiles ? tile_class(ranges[2 * t + 1] - ranges[2 * t]) : 0xffffffffu;
  const uint32_t peers = __match_any_sync(0xffffffffu, c);
  const int leader = __ffs(peers) - 1;
  uint32_t base = 0;
  if ((int)lane == leader && c != 0xffffffffu) base = atomicAdd(&cls_next[c], (uint32_t)__popc(peers));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (c != 0xffffffffu) order[base + __popc(peers & ((1u << lane) - 1u))] = t;
}

void fill_tile_order(const uint32_t* ranges, uint32_t n_tiles, uint32_t* cls, uint32_t* order, cudaStream_t st) {
  const unsigned tb = (n_tiles + 255) / 256;
  if (tb == 0 || cudaMemsetAsync(cls, 0, 256 * sizeof(uint32_t), st) != cudaSuccess) return;  // reported by the caller
  tile_class_count_kernel<<<tb, 256, 0, st>>>(ranges, n_tiles, cls);
  tile_class_starts_kernel<<<1, 256, 0, st>>>(cls);
  tile_order_kernel<<<tb, 256, 0, st>>>(ranges, n_tiles, cls, order);
}

// ---------------------------------------------------------------- planning
inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

struct SortPlan {
  int Tx, Ty, rec_pass, pair_pass, nb_pairs, rec_bps;
  size_t n_items;  // views x n_pad
  size_t off_counts, off_scnt, off_sums, off_rk0, off_rk1, off_rv0, off_rv1, off_keys, off_vals, off_hist, off_hdr,
      off_rows, off_used, off_cls, total;
  uint64_t rows_cap;
};

inline int bits_for(uint64_t v) {  // smallest b with 2^b >= v
  int b = 0;
  while ((1ull << b) < v) ++b;
  return b;
}

SortPlan plan_sort(int32_t n_pad, gs_frame fr, uint64_t capacity) {
  SortPlan p;
  p.Tx = (fr.width + fr.tile_w - 1) / fr.tile_w;
  p.Ty = (fr.height + fr.tile_h - 1) / fr.tile_h;
  const uint64_t tiles = (uint64_t)fr.n_views * p.Tx * p.Ty;
  p.pair_pass = std::max(1, (bits_for(tiles) + 7) / 8);
  p.rec_pass = 4;  // 32 depth bits within each view
  p.n_items = (size_t)fr.n_views * n_pad;
  p.nb_pairs = (int)((capacity + kRadixTile - 1) / kRadixTile);
  p.rec_bps = (int)(((size_t)n_pad + kRadixTile - 1) / kRadixTile);
  const size_t hist_n = (size_t)256 * std::max((size_t)p.nb_pairs, (size_t)fr.n_views * p.rec_bps);
  const size_t sums_n = (size_t)std::max(scan_blocks(p.n_items), scan_blocks(hist_n)) + 1;
  size_t o = 0;
  p.off_counts = o; o += align256(p.n_items * 4);
  p.off_scnt = o;   o += align256(p.n_items * 4);
  p.off_sums = o;   o += align256(sums_n * 4);
  p.off_rk0 = o;    o += align256(p.n_items * 4);
  p.off_rk1 = o;    o += align256(p.n_items * 4);
  p.off_rv0 = o;    o += align256(p.n_items * 4);
  p.off_rv1 = o;    o += align256(p.n_items * 4);
  p.off_keys = o;   o += align256(capacity * 4);
  p.off_vals = o;   o += align256(capacity * 4);
  p.off_hist = o;   o += align256(hist_n * 4);
  p.rows_cap = std::min<uint64_t>(capacity + 2 * (uint64_t)p.n_items, 0xffffffffull);
  p.off_hdr = o;    o += align256(p.n_items * 16);
  p.off_rows = o;   o += align256(p.rows_cap * 8);
  p.off_used = o;   o += 256;
  p.off_cls = o;    o += 256 * 4;
  p.total = o;
  return p;
}

// Stable LSD passes over 8-bit digits starting at `shift0` on nseg segments of
// bpg tiles each (see Seg); the keys/values ping-pong between buffer 0 and 1
// starting in `cur`, which is updated.  The histogram scan runs over
// nseg x 256 x bpg entries, or over the pairs in use when the length is on the
// device.
template <typename K>
void radix_passes(K** kbuf, uint32_t** vbuf, int& cur, int npass, int shift0, Seg sg, int nseg, int bpg,
                  uint32_t* hist, uint32_t* sums, cudaStream_t st) {
  const size_t hist_n = (size_t)nseg * 256 * bpg;
  const unsigned grid = (unsigned)((size_t)nseg * bpg);
  for (int pass = 0; pass < npass; ++pass) {
    const int shift = shift0 + 8 * pass;
    radix_hist_kernel<K><<<grid, kRadixThreads, 0, st>>>(kbuf[cur], sg, bpg, shift, hist);
    exclusive_scan(hist, hist, hist_n, sg.len_dev, sg.cap, sums, nullptr, 0, nullptr, st);
    radix_scatter_kernel<K><<<grid, kRadixThreads, 0, st>>>(kbuf[cur], vbuf[cur], kbuf[cur ^ 1], vbuf[cur ^ 1], sg,
                                                            bpg, shift, hist);
    cur ^= 1;
  }
}

}  // namespace
}  // namespace gs

extern "C" size_t gs_bin_sort_workspace_size(int32_t n_pad, gs_frame frame, uint64_t capacity) {
  if (n_pad < 0 || !gs::frame_ok(frame)) return 0;
  return gs::plan_sort(n_pad, frame, capacity).total;
}

extern "C" gs_status gs_bin_sort(const gs_projected* proj, int32_t n_pad, gs_frame frame, void* workspace,
                                 size_t workspace_bytes, gs_sorted* out, int32_t* status, void* stream) {
  using namespace gs;
  GS_REQUIRE(proj && out && proj->rec, "gs_bin_sort: null argument");
  GS_REQUIRE(out->keys && out->vals && out->ranges && out->n_pairs, "gs_bin_sort: null output buffer");
  GS_REQUIRE(n_pad >= 0 && n_pad % 4 == 0, "gs_bin_sort: bad n_pad=%d", n_pad);
  GS_REQUIRE(frame_ok(frame), "gs_bin_sort: bad frame (tile %dx%d)", frame.tile_w, frame.tile_h);
  GS_REQUIRE(out->capacity > 0 && out->capacity < (1ull << 32), "gs_bin_sort: capacity must be in [1, 2^32)");
  const SortPlan p = plan_sort(n_pad, frame, out->capacity);
  GS_REQUIRE(p.Tx < 65536 && p.Ty < 65536, "gs_bin_sort: at most 65535 tiles per row and column");
  GS_REQUIRE((uint64_t)frame.n_views * p.Tx * p.Ty < 0xffffffffull, "gs_bin_sort: views x tiles must be below 2^32 - 1");
  GS_REQUIRE(workspace && workspace_bytes >= p.total, "gs_bin_sort: workspace needs %zu bytes, got %zu", p.total,
             workspace_bytes);
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  uint32_t* counts = (uint32_t*)(ws + p.off_counts);
  uint32_t* scnt = (uint32_t*)(ws + p.off_scnt);
  uint32_t* sums = (uint32_t*)(ws + p.off_sums);
  uint32_t* hist = (uint32_t*)(ws + p.off_hist);
  const float4* rec = reinterpret_cast<const float4*>(proj->rec);
  const uint64_t T = (uint64_t)p.Tx * p.Ty;

  uint4* hdr = (uint4*)(ws + p.off_hdr);
  uint2* rows = (uint2*)(ws + p.off_rows);
  uint32_t* rows_used = (uint32_t*)(ws + p.off_used);
  if (cudaMemsetAsync(out->ranges, 0, (size_t)frame.n_views * T * 2 * sizeof(uint32_t), st) != cudaSuccess ||
      cudaMemsetAsync(out->n_pairs, 0, sizeof(uint32_t), st) != cudaSuccess ||
      cudaMemsetAsync(rows_used, 0, sizeof(uint32_t), st) != cudaSuccess)
    return check_launch("gs_bin_sort: memset");
  if (p.n_items == 0) {  // no splats: every range is empty
    if (out->order) fill_tile_order(out->ranges, (uint32_t)(frame.n_views * T), (uint32_t*)(ws + p.off_cls), out->order, st);
    return check_launch("gs_bin_sort");
  }
  const int eb = (int)((p.n_items + 255) / 256);
  // records sorted by depth within each view's segment
  uint32_t* rk[2] = {(uint32_t*)(ws + p.off_rk0), (uint32_t*)(ws + p.off_rk1)};
  uint32_t* rv[2] = {(uint32_t*)(ws + p.off_rv0), (uint32_t*)(ws + p.off_rv1)};
  record_keys_kernel<<<eb, 256, 0, st>>>(rec, n_pad, frame, p.Tx, p.Ty, counts, rk[0], rv[0], hdr, rows, p.rows_cap,
                                         rows_used, status);
  int rcur = 0;
  const Seg rseg{nullptr, 0, (uint32_t)n_pad, (uint32_t)n_pad};
  radix_passes<uint32_t>(rk, rv, rcur, p.rec_pass, 0, rseg, frame.n_views, p.rec_bps, hist, sums, st);
  // emission offsets in that order, and the pair count
  gather_counts_kernel<<<eb, 256, 0, st>>>(rv[rcur], counts, scnt, p.n_items);
  exclusive_scan(scnt, scnt, p.n_items, nullptr, 0, sums, out->n_pairs, out->capacity, status, st);
  // pairs in (view, depth, splat) order, then stable passes on their tile keys;
  // the last pass must land in the caller's arrays
  uint32_t* kbuf[2] = {out->keys, (uint32_t*)(ws + p.off_keys)};
  uint32_t* vbuf[2] = {out->vals, (uint32_t*)(ws + p.off_vals)};
  int cur = (p.pair_pass % 2 == 0) ? 0 : 1;
  emit_kernel<<<eb, 256, 0, st>>>(hdr, rows, n_pad, frame, p.Tx, p.Ty, rv[rcur], scnt, out->capacity, kbuf[cur],
                                  vbuf[cur]);
  const Seg pseg{out->n_pairs, out->capacity, 0, 0};
  radix_passes<uint32_t>(kbuf, vbuf, cur, p.pair_pass, 0, pseg, 1, p.nb_pairs, hist, sums, st);
  const int rb = (int)std::min<uint64_t>((out->capacity + 255) / 256, 152 * 16);
  ranges_kernel<<<rb, 256, 0, st>>>(out->keys, out->n_pairs, out->capacity, (uint64_t)frame.n_views * T,
                                    out->ranges);
  if (out->order) fill_tile_order(out->ranges, (uint32_t)(frame.n_views * T), (uint32_t*)(ws + p.off_cls), out->order, st);
  return check_launch("gs_bin_sort");
}
