// qis_block.cuh -- block- and warp-level building blocks shared by the per-search kernels of
// one iteration (qis_iter.cu, qis_scan.cu, qis_merge.cu) and by the fused search kernel
// (qis_search.cu): range and value selection, the near-state test, sorting and merging helpers.
#pragma once
#include "qis_common.cuh"

namespace qis {

constexpr int kSubSites = 64;   // at most this many low-a sites in the bound's subset (2080 candidates)
constexpr int kSubMax = kSubSites * (kSubSites + 1) / 2;

// Block-wide minimum and maximum of one value per thread (every thread gets both).
static __device__ void block_min_max(float& lo, float& hi) {
  __shared__ float s_lo[32], s_hi[32];
  for (int o = 16; o > 0; o >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_lo[w] = lo;
    s_hi[w] = hi;
  }
  __syncthreads();
  lo = s_lo[0];
  hi = s_hi[0];
  for (int k = 1; k < nw; ++k) {
    lo = fminf(lo, s_lo[k]);
    hi = fmaxf(hi, s_hi[k]);
  }
  __syncthreads();
}

// An upper bound of the rank-th smallest (0-based) of cnt values in shared memory, tight to one
// of 256 equal-width bins of the range of the finite ones: the largest value whose bin is at
// most the bin holding that element (binning is monotone, so at least rank + 1 values lie in
// those bins). +inf values (excluded candidates) go to the last bin, so the bound is +inf when
// fewer than rank + 1 values are finite. Two passes over the values instead of the four of a
// radix select. Every thread of the block calls it.
// lo, hi: this thread's minimum and maximum of the finite values (the caller tracks them while
// writing the values; the block-wide range is reduced here).
static __device__ float value_select_upper(const float* v, int cnt, int rank, int* hist, float lo, float hi) {
  __shared__ int s_b;
  for (int t = threadIdx.x; t < 256; t += blockDim.x) hist[t] = 0;
  block_min_max(lo, hi);
  const float scale = 255.99f / fmaxf(hi - lo, 1e-30f);
  for (int t0 = 0; t0 < cnt; t0 += blockDim.x) {
    const int t = t0 + threadIdx.x;
    const bool in = t < cnt;
    const unsigned act = __ballot_sync(0xffffffffu, in);
    if (in) {
      const float x = v[t];
      const int bin = (x <= hi) ? min(255, (int)((x - lo) * scale)) : 255;   // +inf (excluded): last bin
      const unsigned peers = __match_any_sync(act, bin);
      if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&hist[bin], __popc(peers));
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    int b, within;
    find_bin(hist, rank, b, within);
    if (threadIdx.x == 0) s_b = b;
  }
  __syncthreads();
  const int bsel = s_b;
  float mx = -INFINITY, dummy = INFINITY;
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
    const float x = v[t];
    if (((x <= hi) ? min(255, (int)((x - lo) * scale)) : 255) <= bsel) mx = fmaxf(mx, x);
  }
  block_min_max(dummy, mx);
  return mx;
}

// Candidate index of the kept state x if it is one or two flips from the parent p (the single
// flip of its differing site, or the pair of its two), else -1. The words are compared in
// order, four loads in flight per step, and the test stops at the third differing bit: most
// kept states differ in more sites, so most tests read only their first words, while a state
// that is near (the parent itself among them) costs a round trip per four words instead of one
// per word (a rolled loop over the four: a small body fetches better than all W in flight).
static __device__ __forceinline__ long long near_code_sp(const uint64_t* x, const uint64_t* p, int W, int n) {
  int dist = 0, q0 = 0, q1 = 0;
#pragma unroll 1
  for (int w = 0; w < W; w += 4) {
    const uint64_t x0 = x[w];
    const uint64_t x1 = (w + 1 < W) ? x[w + 1] : 0ull;
    const uint64_t x2 = (w + 2 < W) ? x[w + 2] : 0ull;
    const uint64_t x3 = (w + 3 < W) ? x[w + 3] : 0ull;
    uint64_t v = x0 ^ p[w];
    uint64_t v1 = (w + 1 < W) ? (x1 ^ p[w + 1]) : 0ull;
    uint64_t v2 = (w + 2 < W) ? (x2 ^ p[w + 2]) : 0ull;
    uint64_t v3 = (w + 3 < W) ? (x3 ^ p[w + 3]) : 0ull;
#pragma unroll 1
    for (int u = 0; u < 4; ++u) {   // word w + u in v
      while (v) {
        const int pos = (w + u) * 64 + __ffsll((long long)v) - 1;
        if (dist == 0) q0 = pos; else q1 = pos;
        ++dist;
        v &= v - 1;
        if (dist > 2) return -1;
      }
      v = v1;
      v1 = v2;
      v2 = v3;
      v3 = 0ull;
    }
  }
  if (dist == 1) return q0;
  if (dist == 2) return pair_index(n, q0, q1);
  return -1;
}

// The same test for wide states (the per-kernel form, n above 1024): the words are loaded ten at
// a time (one round trip per ten words) and the test stops after the batch that holds the third
// differing bit.
static __device__ __forceinline__ long long near_code_batched(const uint64_t* x, const uint64_t* p, int W, int n) {
  int dist = 0, p0 = 0, p1 = 0;
  for (int w0 = 0; w0 < W; w0 += 10) {
    uint64_t xw[10];
#pragma unroll
    for (int u = 0; u < 10; ++u) xw[u] = (w0 + u < W) ? x[w0 + u] : 0ull;
#pragma unroll
    for (int u = 0; u < 10; ++u) {
      uint64_t v = (w0 + u < W) ? (xw[u] ^ p[w0 + u]) : 0ull;
      if (v && dist < 2) {
        const int lo = (w0 + u) * 64 + __ffsll((long long)v) - 1;
        if (dist == 0) {
          p0 = lo;
          const uint64_t r = v & (v - 1);
          if (r) p1 = (w0 + u) * 64 + __ffsll((long long)r) - 1;
        } else {
          p1 = lo;
        }
      }
      dist += __popcll(v);
    }
    if (dist > 2) return -1;
  }
  if (dist == 1) return p0;
  if (dist == 2) return pair_index(n, p0, p1);
  return -1;
}

constexpr uint32_t kNoCand = 0xffffffffu;   // empty slot of the duplicate table
static __device__ inline uint32_t chash(uint32_t c) { return (c * 2654435761u) >> 7; }



// exclusive prefix sum of one int per thread over the block (blockDim multiple of 32)
static __device__ int block_exclusive_sum(int v, int* wsum /* [33] */, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = (lane < nw) ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) wsum[lane] = w;   // inclusive warp totals
  }
  __syncthreads();
  const int before = (warp > 0 ? wsum[warp - 1] : 0) + x - v;
  *total = wsum[nw - 1];
  __syncthreads();
  return before;
}

// (key, c) order of candidates: energy key, ties by candidate index c (the Alg. 3 loop order).
static __device__ __forceinline__ bool kc_less(unsigned long long ka, unsigned long long ea, unsigned long long kb,
                                        unsigned long long eb) {
  return ka < kb || (ka == kb && (uint32_t)ea < (uint32_t)eb);
}

// Ascending bitonic sort of n2 (power of two) (key, entry) pairs in shared memory, any size.
static __device__ void bitonic_sort_smem(unsigned long long* key, unsigned long long* ent, int n2) {
  for (int k = 2; k <= n2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < n2; t += blockDim.x) {
        const int u = t ^ j;
        if (u > t) {
          const unsigned long long a = key[t], c = key[u], va = ent[t], vc = ent[u];
          const bool up = (t & k) == 0;
          if (kc_less(c, vc, a, va) == up) {
            key[t] = c; key[u] = a;
            ent[t] = vc; ent[u] = va;
          }
        }
      }
      __syncthreads();
    }
  }
}

// Ascending bitonic sort of the 32 (key, entry) pairs of one warp, one per lane, in shuffles.
static __device__ __forceinline__ void warp_sort32(unsigned long long& key, unsigned long long& ent) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const unsigned long long ko = __shfl_xor_sync(0xffffffffu, key, j);
      const unsigned long long eo = __shfl_xor_sync(0xffffffffu, ent, j);
      const bool want_min = ((lane & j) == 0) == ((lane & k) == 0);
      const bool take = want_min ? kc_less(ko, eo, key, ent) : kc_less(key, ent, ko, eo);
      if (take) {
        key = ko;
        ent = eo;
      }
    }
  }
}

// Sort of nv <= blockDim.x pairs: every warp sorts a run of 32 (padding ~0 sorts last), then
// each element's place = its index in its run + the number of smaller elements in every other
// run (binary search, 32 entries). Input in (key, ent)[0..nv), output in (okey, oent)[0..nv).
// Every thread of the block calls it.
static __device__ void sort_runs(const unsigned long long* key, const unsigned long long* ent, int nv,
                          unsigned long long* okey, unsigned long long* oent) {
  const int t = threadIdx.x, w = t >> 5;
  const int nr = (nv + 31) >> 5;
  unsigned long long k = ~0ull, e = ~0ull;
  if (t < nv) {
    k = key[t];
    e = ent[t];
  }
  if (w < nr) warp_sort32(k, e);   // warp-uniform
  okey[t] = k;                     // runs staged in the output arrays (blockDim.x entries)
  oent[t] = e;
  __syncthreads();
  int pos = t & 31;
  const bool real = w < nr && k != ~0ull;   // a finite energy's key is never all ones
  if (real) {
    for (int v = 0; v < nr; ++v) {
      if (v == w) continue;
      const unsigned long long* rk = okey + 32 * v;
      const unsigned long long* re = oent + 32 * v;
      int lo = 0, hi = 32;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (kc_less(rk[mid], re[mid], k, e)) lo = mid + 1; else hi = mid;
      }
      pos += lo;
    }
  }
  __syncthreads();   // every search done before the runs are overwritten
  if (real) {
    okey[pos] = k;
    oent[pos] = e;
  }
  __syncthreads();
}

// Ascending bitonic sort of 32 single keys of one warp, one per lane, in shuffles.
static __device__ __forceinline__ void warp_sort32_key(unsigned long long& key) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const unsigned long long ko = __shfl_xor_sync(0xffffffffu, key, j);
      const bool want_min = ((lane & j) == 0) == ((lane & k) == 0);
      key = want_min ? min(key, ko) : max(key, ko);
    }
  }
}

// sort_runs for packed keys ((key - kmin) << cb | c: one 64-bit value carries the (key, c)
// order when the keys span less than 2^(64 - cb)); the packing is done on load. Output in
// okey[0..nv). Every thread of the block calls it; nv <= blockDim.x.
static __device__ void sort_runs_packed(const unsigned long long* key, const unsigned long long* ent, int nv,
                                 unsigned long long kmin, int cb, unsigned long long* okey) {
  const int t = threadIdx.x, w = t >> 5;
  const int nr = (nv + 31) >> 5;
  unsigned long long k = ~0ull;
  if (t < nv) k = ((key[t] - kmin) << cb) | (uint32_t)ent[t];
  if (w < nr) warp_sort32_key(k);   // warp-uniform
  okey[t] = k;
  __syncthreads();
  int pos = t & 31;
  const bool real = w < nr && k != ~0ull;   // a packed key is never all ones (c < 2^cb - 1)
  if (real) {
    for (int v = 0; v < nr; ++v) {
      if (v == w) continue;
      const unsigned long long* rk = okey + 32 * v;
      int lo = 0, hi = 32;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (rk[mid] < k) lo = mid + 1; else hi = mid;
      }
      pos += lo;
    }
  }
  __syncthreads();
  if (real) okey[pos] = k;
  __syncthreads();
}

static __device__ inline uint64_t flip_mask(int x, int i, int j) {
  uint64_t m = 0;
  if ((i >> 6) == x) m ^= 1ull << (i & 63);
  if (j >= 0 && (j >> 6) == x) m ^= 1ull << (j & 63);
  return m;
}

constexpr int kSparseNB = 128;   // buckets of a_j

static __device__ __forceinline__ int sparse_bucket(float x, float lo, float inv) {
  const float f = __fmul_rn(__fsub_rn(x, lo), inv);   // monotone in x; NaN for inf * 0
  return f < (float)kSparseNB ? max(0, (int)f) : kSparseNB - 1;
}


}  // namespace qis
