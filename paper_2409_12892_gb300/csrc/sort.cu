// Device-wide exclusive scans and a stable LSD radix sort of (u32 key, u32 value)
// pairs. They order the tile keys of the rasterizer (Sec. 3.1 "tile-based
// rasterizer"; the keys are sorted by depth, then stably by tile) and the cache
// segments by splat (the paper's sortCacheByGaussians, Sec. 3.3).
//
// All results are deterministic: ties keep their input order.
#include "internal.cuh"

namespace gslm {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;   // 2048 items per block

// Radix passes of 8-bit digits over 4096-item blocks (16 rounds of 32 items per
// warp), or of 9-bit digits over 2048-item blocks where that takes fewer passes
// (the tile keys: 17 bits, two passes instead of three).
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;

template <typename T>
__device__ __forceinline__ unsigned long long as_u64(T v) {
  return (unsigned long long)v;
}

// Sum of each 2048-item tile.
template <typename Tin>
__global__ void k_tile_sums(const Tin* __restrict__ in, long long n, unsigned long long* __restrict__ sums) {
  const long long base = (long long)blockIdx.x * kScanTile;
  unsigned long long s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const long long i = base + threadIdx.x + (long long)k * kScanThreads;
    if (i < n) s += as_u64(in[i]);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ unsigned long long red[kScanThreads / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) t += red[w];
    sums[blockIdx.x] = t;
  }
}

// Exclusive scan of each tile plus the tile's offset. If total != null, the
// last tile also writes the grand total to *total.
template <typename Tin, typename Tout>
__global__ void k_tile_scan(const Tin* __restrict__ in, long long n, const unsigned long long* __restrict__ offs,
                            Tout* __restrict__ out, Tout* __restrict__ total) {
  __shared__ unsigned long long buf[kScanTile];
  __shared__ unsigned long long wsum[kScanThreads / 32];
  const long long base = (long long)blockIdx.x * kScanTile;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int j = threadIdx.x + k * kScanThreads;
    const long long i = base + j;
    buf[j] = i < n ? as_u64(in[i]) : 0ull;
  }
  __syncthreads();
  unsigned long long v[kScanItems];
  unsigned long long run = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = run;
    run += buf[threadIdx.x * kScanItems + k];
  }
  // inclusive warp scan of the per-thread totals
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long inc = run;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  unsigned long long woff = 0;
  for (int w = 0; w < warp; ++w) woff += wsum[w];
  const unsigned long long toff = offs != nullptr ? offs[blockIdx.x] : 0ull;
  const unsigned long long excl = toff + woff + inc - run;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) buf[threadIdx.x * kScanItems + k] = excl + v[k];
  if (total != nullptr && blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanThreads - 1)
    *total = (Tout)(excl + run);
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int j = threadIdx.x + k * kScanThreads;
    const long long i = base + j;
    if (i < n) out[i] = (Tout)buf[j];
  }
}

long long div_up(long long a, long long b) { return (a + b - 1) / b; }

size_t scan_temp_words(long long n) {
  size_t words = 0;
  long long m = div_up(n, kScanTile);
  while (m > 1) {
    words += 2 * (size_t)m;
    m = div_up(m, kScanTile);
  }
  return words + 4;
}

// Exclusive scan of n inputs; out has n + 1 slots (out[n] = total).
template <typename Tin, typename Tout>
cudaError_t scan_impl(const Tin* in, Tout* out, long long n, unsigned long long* temp, cudaStream_t st) {
  if (n <= 0) {
    return cudaMemsetAsync(out, 0, sizeof(Tout), st);
  }
  const long long nb = div_up(n, kScanTile);
  if (nb == 1) {
    { k_tile_scan<Tin, Tout><<<1, kScanThreads, 0, st>>>(in, n, nullptr, out, out + n); note_launch(); }
    return cudaGetLastError();
  }
  unsigned long long* sums = temp;
  unsigned long long* offs = temp + nb;
  { k_tile_sums<Tin><<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, sums); note_launch(); }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = scan_impl<unsigned long long, unsigned long long>(sums, offs, nb, temp + 2 * nb, st);
  if (e != cudaSuccess) return e;
  { k_tile_scan<Tin, Tout><<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, offs, out, out + n); note_launch(); }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------- radix sort
template <int kBits, int kRounds>
__global__ void k_radix_hist(const uint32_t* __restrict__ keys, long long n, int shift, int nblocks,
                             uint32_t* __restrict__ hist) {
  constexpr int kRadix = 1 << kBits, kSortTile = kSortThreads * kRounds;
  __shared__ uint32_t h[kRadix];
  for (int d = threadIdx.x; d < kRadix; d += kSortThreads) h[d] = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * kSortTile;
  for (int k = 0; k < kRounds; ++k) {
    const long long i = base + threadIdx.x + (long long)k * kSortThreads;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & (kRadix - 1)], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += kSortThreads) hist[(long long)d * nblocks + blockIdx.x] = h[d];
}

// Stable scatter of one block. Items are ranked per digit with warp match
// (stable within a warp), then per warp prefix (stable across warps); the block
// is first reordered by digit in shared memory and then written out, so each
// digit's run goes to global memory with coalesced stores. Thread t owns the
// kDPT consecutive digits from t kDPT for the counts' prefix sums.
template <int kBits, int kRounds>
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals, long long n, int shift, int nblocks,
    const uint32_t* __restrict__ offs, uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out) {
  constexpr int kRadix = 1 << kBits, kSortTile = kSortThreads * kRounds, kDPT = kRadix / kSortThreads;
  static_assert(kDPT == 1 || kDPT == 2, "digits per thread");
  __shared__ uint32_t wcnt[kSortWarps][kRadix];
  __shared__ uint32_t goff[kRadix];
  __shared__ uint32_t lstart[kRadix];
  __shared__ uint32_t wsum[kSortWarps];
  __shared__ uint32_t skeys[kSortTile];
  __shared__ uint32_t svals[kSortTile];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < kRadix; d += kSortThreads) {
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) wcnt[w][d] = 0;
    goff[d] = offs[(long long)d * nblocks + blockIdx.x];
  }
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
  const long long bbase = (long long)blockIdx.x * kSortTile;
  const long long wbase = bbase + (long long)warp * (kRounds * 32);
  uint32_t kk[kRounds], vv[kRounds], rk[kRounds];
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    const long long i = wbase + r * 32 + lane;
    const bool ok = i < n;
    const unsigned okmask = __ballot_sync(0xffffffffu, ok);
    kk[r] = ok ? keys[i] : 0u;
    vv[r] = ok ? vals[i] : 0u;
    rk[r] = 0;
    if (ok) {
      const uint32_t d = (kk[r] >> shift) & (kRadix - 1);
      const unsigned peers = __match_any_sync(okmask, d);
      const uint32_t base = wcnt[warp][d];
      rk[r] = base + __popc(peers & lt);
      __syncwarp(okmask);
      if (lane == __ffs(peers) - 1) wcnt[warp][d] = base + __popc(peers);
    }
    __syncwarp();
  }
  __syncthreads();
  // per digit: warp prefixes, and the block's count of the digit
  uint32_t dc[kDPT];
  uint32_t cnt = 0;
#pragma unroll
  for (int q = 0; q < kDPT; ++q) {
    const int d = threadIdx.x * kDPT + q;
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
      const uint32_t c = wcnt[w][d];
      wcnt[w][d] = run;
      run += c;
    }
    dc[q] = run;
    cnt += run;
  }
  // exclusive scan of the digit counts over the block (digits in thread order)
  uint32_t inc = cnt;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  uint32_t woff = 0;
  for (int w = 0; w < warp; ++w) woff += wsum[w];
  {
    uint32_t st = woff + inc - cnt;
#pragma unroll
    for (int q = 0; q < kDPT; ++q) {
      lstart[threadIdx.x * kDPT + q] = st;
      st += dc[q];
    }
  }
  __syncthreads();
  // reorder by digit in shared memory
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    const long long i = wbase + r * 32 + lane;
    if (i < n) {
      const uint32_t d = (kk[r] >> shift) & (kRadix - 1);
      const uint32_t lp = lstart[d] + wcnt[warp][d] + rk[r];
      skeys[lp] = kk[r];
      svals[lp] = vv[r];
    }
  }
  __syncthreads();
  const long long rem = n - bbase;
  const int valid = rem < kSortTile ? (int)rem : kSortTile;
  for (int t = threadIdx.x; t < valid; t += kSortThreads) {
    const uint32_t key = skeys[t];
    const uint32_t d = (key >> shift) & (kRadix - 1);
    const uint32_t pos = goff[d] + (uint32_t)t - lstart[d];
    keys_out[pos] = key;
    vals_out[pos] = svals[t];
  }
}

// ---------------------------------------------------------------------------- small helpers
__global__ void k_compact(const uint32_t* __restrict__ counts, const uint32_t* __restrict__ pos, long long n,
                          uint32_t* __restrict__ list) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && counts[i] > 0) list[pos[i]] = (uint32_t)i;
}

__global__ void k_flags(const uint32_t* __restrict__ counts, long long n, uint32_t* __restrict__ flags) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flags[i] = counts[i] > 0 ? 1u : 0u;
}

__global__ void k_gather(const uint32_t* __restrict__ src, const uint32_t* __restrict__ idx, long long n,
                         uint32_t* __restrict__ dst) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[idx[i]];
}

__global__ void k_scatter_index(const uint32_t* __restrict__ idx, long long n, uint32_t* __restrict__ dst) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[idx[i]] = (uint32_t)i;
}

__global__ void k_iota(uint32_t* __restrict__ dst, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (uint32_t)i;
}

__global__ void k_ranges(const uint32_t* __restrict__ keys, long long n, uint32_t* __restrict__ start,
                         uint32_t* __restrict__ end) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t k = keys[i];
  if (i == 0 || keys[i - 1] != k) start[k] = (uint32_t)i;
  if (i == n - 1 || keys[i + 1] != k) end[k] = (uint32_t)(i + 1);
}

unsigned grid_for(long long n, int bs) { return (unsigned)div_up(n, bs); }

}  // namespace

size_t scan_temp_bytes(long long n) { return scan_temp_words(n) * sizeof(unsigned long long); }

cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, long long n, void* temp, cudaStream_t st) {
  return scan_impl<uint32_t, uint32_t>(in, out, n, static_cast<unsigned long long*>(temp), st);
}

cudaError_t exclusive_scan_u64(const uint32_t* in, unsigned long long* out, long long n, void* temp,
                               cudaStream_t st) {
  return scan_impl<uint32_t, unsigned long long>(in, out, n, static_cast<unsigned long long*>(temp), st);
}

// Histogram words of the larger (9-bit) configuration, which holds the other.
size_t radix_temp_bytes(long long n) {
  const long long nb = div_up(n > 0 ? n : 1, kSortThreads * 8);
  const long long h = nb * 512;
  return (size_t)(2 * h + 1) * sizeof(uint32_t) + scan_temp_bytes(h) + 256;
}

template <int kBits, int kRounds>
cudaError_t radix_passes(uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp, uint32_t* vals_tmp, long long n,
                         int bits, void* temp, uint32_t** keys_out, uint32_t** vals_out, cudaStream_t st) {
  constexpr int kRadix = 1 << kBits;
  const int nblocks = (int)div_up(n, kSortThreads * kRounds);
  const long long h = (long long)nblocks * kRadix;
  uint32_t* hist = static_cast<uint32_t*>(temp);
  uint32_t* offs = hist + h;
  void* scan_tmp = reinterpret_cast<void*>(reinterpret_cast<uintptr_t>(offs + h + 1 + 64) & ~uintptr_t(63));
  uint32_t *ki = keys, *vi = vals, *ko = keys_tmp, *vo = vals_tmp;
  for (int shift = 0; shift < bits; shift += kBits) {
    { k_radix_hist<kBits, kRounds><<<nblocks, kSortThreads, 0, st>>>(ki, n, shift, nblocks, hist); note_launch(); }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = exclusive_scan_u32(hist, offs, h, scan_tmp, st);
    if (e != cudaSuccess) return e;
    {
      k_radix_scatter<kBits, kRounds><<<nblocks, kSortThreads, 0, st>>>(ki, vi, n, shift, nblocks, offs, ko, vo);
      note_launch();
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    uint32_t* t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
  }
  *keys_out = ki;
  *vals_out = vi;
  return cudaSuccess;
}

cudaError_t radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp, uint32_t* vals_tmp, long long n,
                             int bits, void* temp, uint32_t** keys_out, uint32_t** vals_out, cudaStream_t st) {
  *keys_out = keys;
  *vals_out = vals;
  if (n <= 1 || bits <= 0) return cudaSuccess;
  if ((bits + 8) / 9 < (bits + 7) / 8)
    return radix_passes<9, 8>(keys, vals, keys_tmp, vals_tmp, n, bits, temp, keys_out, vals_out, st);
  return radix_passes<8, 16>(keys, vals, keys_tmp, vals_tmp, n, bits, temp, keys_out, vals_out, st);
}

cudaError_t launch_compact_flags(const uint32_t* counts, const uint32_t* pos, long long n, uint32_t* list,
                                 cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  { k_compact<<<grid_for(n, 256), 256, 0, st>>>(counts, pos, n, list); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_flags(const uint32_t* counts, long long n, uint32_t* flags, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  { k_flags<<<grid_for(n, 256), 256, 0, st>>>(counts, n, flags); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_gather_u32(const uint32_t* src, const uint32_t* idx, long long n, uint32_t* dst,
                              cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  { k_gather<<<grid_for(n, 256), 256, 0, st>>>(src, idx, n, dst); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_scatter_index_u32(const uint32_t* idx, long long n, uint32_t* dst, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  { k_scatter_index<<<grid_for(n, 256), 256, 0, st>>>(idx, n, dst); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_iota_u32(uint32_t* dst, long long n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  { k_iota<<<grid_for(n, 256), 256, 0, st>>>(dst, n); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_ranges(const uint32_t* keys, long long n, uint32_t* start, uint32_t* end, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  { k_ranges<<<grid_for(n, 256), 256, 0, st>>>(keys, n, start, end); note_launch(); }
  return cudaGetLastError();
}

}  // namespace gslm
