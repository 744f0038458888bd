// qis_instance.cu -- per-instance preparation, search initialisation and FP64 rescoring.
//
// Instance data (H0 of Eq. (1)) lives in padded n_pad x n_pad planes:
//   J64  FP64 couplings as given (zero padding)
//   Jq   fixed-point couplings Jq = J * 2^q (int64, exact on the 2^-q grid)
//   J4   fl32(4 * Jq * 2^-q): the candidate filter's coupling term
//   D16  Jq written in balanced base-4096 digits, Jq = sum_d 4096^d D_d, D_d in [-2048, 2047],
//        one FP16 plane per digit (every digit is an exact FP16 integer)
#include <algorithm>

#include "qis_common.cuh"

namespace qis {

// ---------------------------------------------------------------- validation
// stats layout (doubles): [0] bad flags (as bits of an int), [1] max frac bits, [2] max|J| bits,
// [3] max|h| bits, [4 .. 4+n) row sums sum_{j>i} |J_ij|; the host adds [4+n] = sum_i |h_i|.
// Fraction bits of x: the smallest f >= 0 with x 2^f an integer, from the bit pattern
// (|x| = M 2^(e - 1075) with the 53-bit significand M for a normal x, m 2^-1074 for a
// subnormal one; the lowest set bit of the significand decides).
__device__ inline int frac_bits(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
  if (u == 0) return 0;
  const int e = (int)(u >> 52);
  const unsigned long long m = u & 0xfffffffffffffull;
  const int fb = (e == 0) ? 1074 - (__ffsll((long long)m) - 1)
                          : 1075 - e - (__ffsll((long long)(m | (1ull << 52))) - 1);
  return fb > 0 ? fb : 0;
}

// One warp per row i (its lanes over the columns, coalesced): finiteness, zero diagonal,
// bitwise symmetry, fraction bits and max |J_ij| (as the bit patterns of non-negative
// doubles, which order as integers), and the row sum of |J_ij|, j > i, reduced in a fixed
// shuffle order (deterministic). Sum of |h| is formed on the host.
__device__ __forceinline__ void validate_row(const double* J64, const double* h64, int n, int n_pad, double* stats, int i) {
  int* bad = reinterpret_cast<int*>(stats);
  int* maxfrac = reinterpret_cast<int*>(stats + 1);
  unsigned long long* maxJ = reinterpret_cast<unsigned long long*>(stats + 2);
  unsigned long long* maxh = reinterpret_cast<unsigned long long*>(stats + 3);
  const int lane = threadIdx.x & 31;
  const double* row = J64 + (long long)i * n_pad;
  double rs = 0.0;
  int fb = 0, b = 0;
  unsigned long long mj = 0;
  for (int j = lane; j < n; j += 32) {
    const double x = row[j];
    const unsigned long long ax = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
    if (ax >= 0x7ff0000000000000ull) b |= 1;   // Inf or NaN
    if (j == i) {
      if (ax != 0) b |= 2;
      continue;
    }
    if (__double_as_longlong(x) != __double_as_longlong(J64[(long long)j * n_pad + i])) b |= 4;
    fb = max(fb, frac_bits(x));
    mj = max(mj, ax);
    if (j > i) rs += fabs(x);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rs += __shfl_xor_sync(0xffffffffu, rs, o);
    fb = max(fb, __shfl_xor_sync(0xffffffffu, fb, o));
    mj = max(mj, __shfl_xor_sync(0xffffffffu, mj, o));
    b |= __shfl_xor_sync(0xffffffffu, b, o);
  }
  if (lane == 0) {
    const double hv = h64[i];
    const unsigned long long ah = (unsigned long long)__double_as_longlong(hv) & 0x7fffffffffffffffull;
    if (ah >= 0x7ff0000000000000ull) b |= 8;
    fb = max(fb, frac_bits(hv));
    stats[4 + i] = rs;
    if (b) atomicOr(bad, b);
    atomicMax(maxfrac, fb);
    atomicMax(maxJ, mj);
    atomicMax(maxh, ah);
  }
}

__global__ void __launch_bounds__(256) k_validate(const double* J64, const double* h64, int n, int n_pad, double* stats) {
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= n) return;   // warp-uniform
  validate_row(J64, h64, n, n_pad, stats, i);
}

// A batch of instances at once: blockIdx.y is the instance of the batch (its layout item).
__global__ void __launch_bounds__(256) k_validate_batch(const LayoutItem* items, const double* J64, const double* h64) {
  const LayoutItem L = items[blockIdx.y];
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= L.n) return;   // warp-uniform
  validate_row(J64 + L.off_mat, h64 + L.off_vec, L.n, L.n_pad, L.stats, i);
}

cudaError_t launch_validate(const DevPtrs& P, int inst, int n, long long off_mat, long long off_vec,
                            double* stats, cudaStream_t s) {
  (void)inst;
  cudaMemsetAsync(stats, 0, 4 * sizeof(double), s);
  const int np = pad_of(n);
  k_validate<<<(n + 7) / 8, 256, 0, s>>>(P.J64 + off_mat, P.h64 + off_vec, n, np, stats);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- padded layout
// J (n x n, contiguous, as copied from the host) into the padded n_pad x n_pad plane; zeros
// past n.
__global__ void k_restride(const double* src, int n, int n_pad, double* dst) {
  const long long total = (long long)n_pad * n_pad;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / n_pad), j = (int)(e % n_pad);
    dst[e] = (i < n && j < n) ? src[(long long)i * n + j] : 0.0;
  }
}

// Rows i = blockIdx.x, blockIdx.x + gridDim.x, ... of every instance (blockIdx.y), the threads
// over the columns: coalesced reads of the caller's rows (page-locked host memory read in place
// where it is), no index division.
__global__ void k_restride_batch(const LayoutItem* items, double* J64) {
  const LayoutItem L = items[blockIdx.y];
  double* dst = J64 + L.off_mat;
  for (int i = blockIdx.x; i < L.n_pad; i += gridDim.x) {
    const double* src = L.src + (long long)i * L.n;
    double* row = dst + (long long)i * L.n_pad;
    for (int j = threadIdx.x; j < L.n_pad; j += blockDim.x) row[j] = (i < L.n && j < L.n) ? src[j] : 0.0;
  }
}

// Layout and validation of `count` staged instances (items on the device), two launches.
cudaError_t launch_layout_batch(const DevPtrs& P, const LayoutItem* items, int count, int max_n_pad, double* J64,
                                cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_restride_batch<<<dim3(max_n_pad, count), 256, 0, s>>>(items, J64);
  k_validate_batch<<<dim3((max_n_pad + 7) / 8, count), 256, 0, s>>>(items, P.J64, P.h64);
  return cudaGetLastError();
}

cudaError_t launch_restride(const double* src, int n, int n_pad, double* dst, cudaStream_t s) {
  const long long total = (long long)n_pad * n_pad;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 4096);
  k_restride<<<blocks, 256, 0, s>>>(src, n, n_pad, dst);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- fixed point + digits
// D16 holds, per digit and instance, an NP x NP plane in the tiled layout of d16_offset.
__global__ void k_quantize(const double* J64, const double* h64, int n, int n_pad, int NP, int q, int digits,
                           int dbits, long long plane, __half* D16, long long* Jq, float* J4, long long* hq) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long tot = (long long)n_pad * n_pad;
  if (e < tot) {
    const int i = (int)(e / n_pad), j = (int)(e % n_pad);
    long long v = 0;
    if (i < n && j < n) v = __double2ll_rn(ldexp(J64[e], q));
    Jq[e] = v;
    J4[e] = (float)(4.0 * ldexp((double)v, -q));
    long long x = v;
    const long long base = 1ll << dbits;
    for (int d = 0; d < digits; ++d) {
      long long r = x & (base - 1);           // x mod base
      if (r >= base / 2) r -= base;           // balanced digit in [-base/2, base/2)
      D16[d * plane + d16_offset(i, j, NP)] = __float2half_rn((float)r);
      x = (x - r) >> dbits;                   // exact
    }
  }
  if (e < n_pad) hq[e] = (e < n) ? __double2ll_rn(ldexp(h64[e], q)) : 0;
}

// x 2^q rounded to the nearest integer, ties to even (what __double2ll_rn(ldexp(x, q)) gives),
// from the bit pattern of x with integer operations only (GB300's FP64 pipe is narrow). x is
// finite (validated) and |x 2^q| < 2^62 (the grid is chosen so).
__device__ __forceinline__ long long fixed_point_rn(double x, int q) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((u >> 52) & 0x7ff);
  unsigned long long m = u & 0xfffffffffffffull;
  if (e == 0 && m == 0) return 0;
  if (e != 0) m |= 1ull << 52;                    // normal: the implicit bit
  const int sh = (e == 0 ? 1 : e) - 1075 + q;     // |x| 2^q = m 2^sh
  long long v;
  if (sh >= 0) {
    v = (long long)(m << sh);
  } else if (sh <= -54) {
    v = 0;   // below 1/2
  } else {
    const int r = -sh;
    const unsigned long long t = m >> r, rem = m & ((1ull << r) - 1), half = 1ull << (r - 1);
    v = (long long)(t + ((rem > half || (rem == half && (t & 1ull))) ? 1ull : 0ull));
  }
  return (u >> 63) ? -v : v;
}

// Instances first .. first+count-1 at once (blockIdx.y), descriptors read on the device; rows
// i = blockIdx.x, blockIdx.x + gridDim.x, ..., the threads over the columns (no index division).
// Jq = rn(J 2^q), J4 = fl32(4 Jq 2^-q) (= fl32(Jq) 2^(2-q): scaling by a power of two commutes
// with rounding), the balanced base-2^dbits digits of Jq.
__global__ void k_quantize_batch(DevPtrs P, int first, __half* D16, long long* Jq, float* J4, long long* hq) {
  const int inst = first + blockIdx.y;
  const InstDesc d = P.inst[inst];
  const double* J64 = P.J64 + d.off_mat;
  __half* D = D16 + (long long)inst * P.NP * P.NP;
  const long long base = 1ll << d.dbits;
  const bool wide_q = d.q > 120;   // 2^(2-q) below the normal floats (tiny couplings): FP64 path
  const float s4 = wide_q ? 0.f : __int_as_float((127 + 2 - d.q) << 23);   // 2^(2-q)
  for (int i = blockIdx.x; i < d.n_pad; i += gridDim.x) {
    for (int j = threadIdx.x; j < d.n_pad; j += blockDim.x) {
      const long long e = (long long)i * d.n_pad + j;
      long long v = 0;
      if (i < d.n && j < d.n) v = fixed_point_rn(J64[e], d.q);
      Jq[d.off_mat + e] = v;
      J4[d.off_mat + e] = wide_q ? (float)(4.0 * ldexp((double)v, -d.q)) : __ll2float_rn(v) * s4;
      long long x = v;
      for (int dg = 0; dg < d.digits; ++dg) {
        long long r = x & (base - 1);           // x mod base
        if (r >= base / 2) r -= base;           // balanced digit in [-base/2, base/2)
        D[dg * P.pool_mat + d16_offset(i, j, P.NP)] = __float2half_rn((float)(int)r);
        x = (x - r) >> d.dbits;                 // exact
      }
    }
  }
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d.n_pad; e += gridDim.x * blockDim.x)
    hq[d.off_vec + e] = (e < d.n) ? __double2ll_rn(ldexp(P.h64[d.off_vec + e], d.q)) : 0;
}

__global__ void __launch_bounds__(256) k_rowmax4_batch(DevPtrs P, int first) {
  const InstDesc d = P.inst[first + blockIdx.y];
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= d.n_pad) return;   // warp-uniform
  const float* J4 = P.J4 + d.off_mat;
  float m = 0.f;
  if (i < d.n)
    for (int j = lane; j < d.n; j += 32) m = fmaxf(m, fabsf(J4[(long long)i * d.n_pad + j]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) P.rm4[d.off_vec + i] = m;
}

// Fixed-point planes, digits and row maxima of instances first .. first+count-1, two launches.
cudaError_t launch_prepare_batch(const DevPtrs& P, int first, int count, int max_n_pad, __half* D16, long long* Jq,
                                 float* J4, long long* hq, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_quantize_batch<<<dim3(max_n_pad, count), 256, 0, s>>>(P, first, D16, Jq, J4, hq);
  k_rowmax4_batch<<<dim3((max_n_pad + 7) / 8, count), 256, 0, s>>>(P, first);
  return cudaGetLastError();
}

cudaError_t launch_quantize(const DevPtrs& P, const InstDesc& d, int inst, __half* D16, long long* Jq,
                            float* J4, long long* hq, cudaStream_t s) {
  const long long tot = (long long)d.n_pad * d.n_pad;
  k_quantize<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
      P.J64 + d.off_mat, P.h64 + d.off_vec, d.n, d.n_pad, P.NP, d.q, d.digits, d.dbits, P.pool_mat,
      D16 + (long long)inst * P.NP * P.NP, Jq + d.off_mat, J4 + d.off_mat, hq + d.off_vec);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- row maxima of the filter couplings
// rm4_i = max_j |4J~_ij| (the FP32 couplings of the scan), a warp per row.
__global__ void __launch_bounds__(256) k_rowmax4(const float* J4, int n, int n_pad, float* rm4) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= n_pad) return;   // warp-uniform
  float m = 0.f;
  if (i < n)
    for (int j = lane; j < n; j += 32) m = fmaxf(m, fabsf(J4[(long long)i * n_pad + j]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) rm4[i] = m;
}

cudaError_t launch_rowmax4(const DevPtrs& P, const InstDesc& d, cudaStream_t s) {
  k_rowmax4<<<(d.n_pad + 7) / 8, 256, 0, s>>>(P.J4 + d.off_mat, d.n, d.n_pad, P.rm4 + d.off_vec);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- search initialisation
// Alg. 3 initial list: [psi0, K placeholders], E(psi0) from Eq. (1), nothing used.
// mode 1 (cached): E(psi0) is taken from init_E / init_q, written by k_init_energy (split modes:
// exact int64 E 2^q, several states per block) or by an earlier launch for the same initial
// states. Mode 2 (deferred, split modes): E(psi0) is left to the first iteration of the fused
// search kernel, which forms it from the exact fields of psi0 that the iteration computes anyway;
// the entry holds 0 until then and e0_pend marks the search. Mode 0 (FP64 mode): one thread adds
// the pair terms i-major, j ascending, then the field terms.
__global__ void __launch_bounds__(256) k_init_search(DevPtrs P, int b0, int mode) {
  const bool cached = mode == 1;
  const int b = b0 + blockIdx.x;
  const InstDesc d = P.inst[b / P.R];
  const int n = d.n, np = d.n_pad, W = d.W;
  __shared__ uint64_t bits[kMaxN / 64];
  __shared__ long long red[1];
  for (int w = threadIdx.x; w < W; w += blockDim.x) bits[w] = P.init_bits[(long long)b * P.Wmax + w];
  __syncthreads();
  double E0 = 0.0;
  if (cached) {
    E0 = P.init_E[b];
    if (threadIdx.x == 0) red[0] = P.init_q[b];
  } else if (mode == 2) {
    if (threadIdx.x == 0) red[0] = 0;
  } else if (threadIdx.x == 0) {
    double Pp = 0.0, F = 0.0;
    const double* J = P.J64 + d.off_mat;
    for (int i = 0; i < n; ++i) {
      const double si = sigma_of(bits, i) ? -1.0 : 1.0;
      for (int j = i + 1; j < n; ++j) {
        const double sj = sigma_of(bits, j) ? -1.0 : 1.0;
        Pp = __dadd_rn(Pp, J[(long long)i * np + j] * si * sj);
      }
    }
    for (int i = 0; i < n; ++i) F = __dadd_rn(F, P.h64[d.off_vec + i] * (sigma_of(bits, i) ? -1.0 : 1.0));
    E0 = __dadd_rn(Pp, F);
    red[0] = 0;
  }
  // Zobrist hash of psi0: XOR over the threads' sites, then over the warps
  __shared__ uint64_t s_h[8];
  uint64_t hsh = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (sigma_of(bits, i)) hsh ^= P.zob[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) hsh ^= __shfl_xor_sync(0xffffffffu, hsh, o);
  if ((threadIdx.x & 31) == 0) s_h[threadIdx.x >> 5] = hsh;
  const long long base = (long long)b * P.K1;
  for (int w = threadIdx.x; w < W; w += blockDim.x) P.lst_bits[base * P.Wmax + w] = bits[w];
  for (int k = threadIdx.x; k < P.K1; k += blockDim.x) {
    P.lst_used[base + k] = 0;
    P.lst_ord[base + k] = (k == 0) ? 0 : -1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) hsh ^= s_h[w];
    P.init_E[b] = E0;
    P.init_q[b] = (P.mode != QIS_FP64) ? red[0] : 0;
    P.lst_E[base] = E0;
    if (P.mode != QIS_FP64) P.lst_q[base] = red[0];
    P.lst_key[base] = (P.mode != QIS_FP64) ? qkey(red[0]) : dkey(E0);
    P.lst_stamp[base] = 0;
    P.lst_hash[base] = hsh;
    P.lst_count[b] = 1;
    P.active[b] = 1;
    P.iter_t[b] = 0;
    if (P.ring_t0) P.ring_t0[b] = 0;
    P.surv_cnt[b] = 0;
    P.e0_pend[b] = mode == 2;
  }
}

cudaError_t launch_init_search(const DevPtrs& P, int b0, int nb, cudaStream_t s, bool cached, bool deferred) {
  if (nb <= 0) return cudaSuccess;
  k_init_search<<<nb, 256, 0, s>>>(P, b0, deferred ? 2 : cached ? 1 : 0);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- rescoring from scratch
// E = sum_{i<j} J_ij s_i s_j + sum_i h_i s_i (Eq. 1) of up to kRG states of one instance per
// block of 256 threads. With x_ij = 1 where s_i != s_j (s = -1 where the bit is set),
// s_i s_j = 1 - 2 x_ij and s_i = 1 - 2 sigma_i, so
//   E = Q - 2 P,  Q = sum_{i<j} J_ij + sum_i h_i,  P = sum_{i<j, x_ij = 1} J_ij + sum_{sigma_i = 1} h_i:
// one pass over the upper triangle serves every state of the block. mask[j] holds the block's
// spins of site j as bits; a coupling loaded once is added to the accumulator of every state
// whose two spins differ. Warp w takes rows w, w + 8, ... of the block's row range, its lanes the
// columns j > i (coalesced). T = long long: the exact fixed-point couplings Jq, hq of an instance
// on its grid 2^-q (every summation order gives the same integer); T = double: the FP64
// couplings, summed in an order fixed by the block shape and not by the state's place in the
// group. When there are few groups (large n, few states), the rows are split over `parts`
// blocks per group, whose partial sums a second kernel adds in part order (the FP64 form takes a
// number of parts fixed by n alone, so every call forms a state's energy the same way).
constexpr int kRG = 16;

// Rows [i0, i1) of the upper triangle (and the h terms if with_h): red[g] = P_g, red[kRG] = Q.
template <typename T>
__device__ void rescore_part(const T* __restrict__ Jm, const T* __restrict__ hv, int n, int n_pad, int i0, int i1,
                             bool with_h, const uint16_t* __restrict__ mask, T* red /* [9][kRG + 1] */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T q = 0, p[kRG];
#pragma unroll
  for (int g = 0; g < kRG; ++g) p[g] = 0;
  for (int i = i0 + warp; i < i1; i += 8) {
    const T* __restrict__ row = Jm + (long long)i * n_pad;
    const unsigned mi = mask[i];
#pragma unroll 2
    for (int j = i + 1 + lane; j < n; j += 32) {
      const T v = row[j];
      const unsigned x = mi ^ mask[j];
      q += v;
#pragma unroll
      for (int g = 0; g < kRG; ++g)
        if ((x >> g) & 1u) p[g] += v;
    }
  }
  if (with_h)
    for (int i = threadIdx.x; i < n; i += 256) {
      const T v = hv[i];
      const unsigned m = mask[i];
      q += v;
#pragma unroll
      for (int g = 0; g < kRG; ++g)
        if ((m >> g) & 1u) p[g] += v;
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    q += __shfl_xor_sync(0xffffffffu, q, o);
#pragma unroll
    for (int g = 0; g < kRG; ++g) p[g] += __shfl_xor_sync(0xffffffffu, p[g], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int g = 0; g < kRG; ++g) red[warp * (kRG + 1) + g] = p[g];
    red[warp * (kRG + 1) + kRG] = q;
  }
  __syncthreads();
  if (threadIdx.x <= kRG) {
    T t = 0;
    for (int w = 0; w < 8; ++w) t += red[w * (kRG + 1) + threadIdx.x];
    red[8 * (kRG + 1) + threadIdx.x] = t;
  }
  __syncthreads();
  if (threadIdx.x <= kRG) red[threadIdx.x] = red[8 * (kRG + 1) + threadIdx.x];
  __syncthreads();
}

// First row of part b of `parts` row ranges with about equal shares of the triangle (rows i..n-1
// hold (n - i)^2 / 2 of its pairs): n - round(n sqrt(1 - b / parts)); part 0 starts at row 0.
__device__ inline int part_row(int n, int b, int parts) {
  if (b <= 0) return 0;
  if (b >= parts) return n;
  const int r = n - (int)lrintf((float)n * sqrtf(1.f - (float)b / (float)parts));
  return min(max(r, 0), n);
}

constexpr int kRPmax = 32;   // row parts per group at most

// Rows of part blockIdx.y of `parts`, then E of the group's states (one part), or their partial
// sums (P, Q) into part[(g * PS + blockIdx.y) * 2 ...] for the states g = 0 .. cnt - 1 of the
// group (several parts; PS >= parts, the stride of one state). Calls out(g, E) for g < cnt in the
// first case.
template <typename T, typename Out>
__device__ void rescore_group(const T* Jm, const T* hv, int n, int n_pad, const uint16_t* mask, T* red, int cnt,
                              int parts, T* part, int PS, Out out) {
  const int b = blockIdx.y;
  rescore_part<T>(Jm, hv, n, n_pad, part_row(n, b, parts), part_row(n, b + 1, parts), b == 0, mask, red);
  if (threadIdx.x < cnt) {
    if (parts == 1) {
      out((int)threadIdx.x, red[kRG] - 2 * red[threadIdx.x]);
    } else {
      T* x = part + ((long long)threadIdx.x * PS + b) * 2;
      x[0] = red[threadIdx.x];
      x[1] = red[kRG];
    }
  }
}

// E = Q - 2 P of a state from its `parts` partial sums (stride 2 between parts), added in order.
template <typename T>
__device__ inline T rs_energy(const T* part, int parts) {
  T p = 0, q = 0;
  for (int b = 0; b < parts; ++b) {
    p += part[2 * b];
    q += part[2 * b + 1];
  }
  return q - 2 * p;
}

// The spin masks of cnt <= kRG states (their words at src[g], Wn words each) into mask[0..n).
__device__ void group_masks(const uint64_t* const* src, int cnt, int n, uint16_t* mask) {
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    unsigned m = 0;
    for (int g = 0; g < cnt; ++g) m |= (unsigned)((src[g][j >> 6] >> (j & 63)) & 1ull) << g;
    mask[j] = (uint16_t)m;
  }
}

// Row parts of the FP64 form: a number fixed by n alone, so that a state's energy is summed the
// same way whichever call and group rescore it.
__host__ __device__ inline int fp64_parts(int n) { return n / 512 < 1 ? 1 : (n / 512 > kRPmax ? kRPmax : n / 512); }

// Row parts per group. Exact form: one unless the groups alone leave the SMs idle (any split
// gives the same integers). FP64 form: fp64_parts(n).
int rescore_parts(const DevPtrs& P, int groups, int n, bool exact) {
  if (!exact) return fp64_parts(n);
  if (groups <= 0) return 1;
  const int target = 4 * (P.sms > 0 ? P.sms : 148);
  int parts = (target + groups - 1) / groups;
  parts = std::min(std::min(parts, kRPmax), std::max(1, n / 256));
  return std::max(parts, 1);
}

// Energies of `count` states (Wn words each, consecutive) of one instance: block x takes
// states kRG x ... kRG x + kRG - 1, block y its part of the rows.
template <typename T>
__global__ void __launch_bounds__(256) k_rescore(const T* Jm, const T* hv, int n, int n_pad, double scale,
                                                 const uint64_t* states, int Wn, int count, double* E_out,
                                                 unsigned long long* acc) {
  extern __shared__ __align__(16) unsigned char rsm[];
  T* red = reinterpret_cast<T*>(rsm);
  uint16_t* mask = reinterpret_cast<uint16_t*>(red + 9 * (kRG + 1));
  __shared__ const uint64_t* src[kRG];
  const int g0 = blockIdx.x * kRG, cnt = min(kRG, count - g0);
  if (threadIdx.x < kRG) src[threadIdx.x] = states + (long long)(g0 + min((int)threadIdx.x, cnt - 1)) * Wn;
  __syncthreads();
  group_masks(src, cnt, n, mask);
  __syncthreads();
  rescore_group<T>(Jm, hv, n, n_pad, mask, red, cnt, gridDim.y, reinterpret_cast<T*>(acc) + 2ll * g0 * gridDim.y,
                   gridDim.y, [&](int g, T E) { E_out[g0 + g] = (double)E * scale; });
}

template <typename T>
__global__ void k_rescore_finish(const unsigned long long* acc, int count, int parts, double scale, double* E_out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < count) E_out[s] = (double)rs_energy(reinterpret_cast<const T*>(acc) + 2ll * s * parts, parts) * scale;
}

size_t rescore_smem(int n, int bytes_T) { return (size_t)9 * (kRG + 1) * bytes_T + (size_t)n * 2; }

cudaError_t launch_rescore(const DevPtrs& P, const InstDesc& d, const uint64_t* bits, int count, int Wn,
                           double* E_out, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const int groups = (count + kRG - 1) / kRG;
  const size_t sm = rescore_smem(d.n, 8);
  const bool exact = P.mode != QIS_FP64 && !d.rounded;
  const int parts = rescore_parts(P, groups, d.n, exact);
  if (exact) {
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_rescore<long long>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_rescore<long long><<<dim3(groups, parts), 256, sm, s>>>(P.Jq + d.off_mat, P.hq + d.off_vec, d.n, d.n_pad,
                                                              d.inv_scale, bits, Wn, count, E_out, P.rs_acc);
    if (parts > 1)
      k_rescore_finish<long long><<<(count + 255) / 256, 256, 0, s>>>(P.rs_acc, count, parts, d.inv_scale, E_out);
  } else {
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_rescore<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_rescore<double><<<dim3(groups, parts), 256, sm, s>>>(P.J64 + d.off_mat, P.h64 + d.off_vec, d.n, d.n_pad, 1.0,
                                                           bits, Wn, count, E_out, P.rs_acc);
    if (parts > 1) k_rescore_finish<double><<<(count + 255) / 256, 256, 0, s>>>(P.rs_acc, count, parts, 1.0, E_out);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- merged-list gather
__global__ void k_gather_merged(DevPtrs P, int inst, int k, int Wn, uint64_t* out) {
  const int r = blockIdx.x;
  if (r >= k) return;
  const int ref = P.mrg_ref[inst * P.K1 + r];
  const int b = ref / P.K1, slot = ref % P.K1;
  for (int w = threadIdx.x; w < Wn; w += blockDim.x)
    out[(long long)r * Wn + w] = P.lst_bits[((long long)b * P.K1 + slot) * P.Wmax + w];
}

cudaError_t launch_gather_merged(const DevPtrs& P, int inst, const InstDesc& d, int k, uint64_t* bits_out,
                                 cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  k_gather_merged<<<k, 32, 0, s>>>(P, inst, k, d.W, bits_out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- initial energies
// E(psi0) 2^q of the initial states of instances inst0, inst0 + 1, ... in the split modes
// (exact int64, Eq. 1), kRG states of one instance per block (row parts as above), into
// init_q / init_E; the search initialisation then takes them as cached values.
__device__ inline void init_energy_out(const DevPtrs& P, const InstDesc& d, long long b, long long Eq) {
  P.init_q[b] = Eq;
  P.init_E[b] = ldexp((double)Eq, -d.q);
}

__global__ void __launch_bounds__(256) k_init_energy(DevPtrs P, int inst0, int ng) {
  const int inst = inst0 + blockIdx.x / ng, g0 = (blockIdx.x % ng) * kRG;
  const int cnt = min(kRG, P.R - g0);
  const InstDesc d = P.inst[inst];
  extern __shared__ __align__(16) unsigned char rsm[];
  long long* red = reinterpret_cast<long long*>(rsm);
  uint16_t* mask = reinterpret_cast<uint16_t*>(red + 9 * (kRG + 1));
  __shared__ const uint64_t* src[kRG];
  const long long b0 = (long long)d.first_search + g0;
  if (threadIdx.x < kRG) src[threadIdx.x] = P.init_bits + (b0 + min((int)threadIdx.x, cnt - 1)) * P.Wmax;
  __syncthreads();
  group_masks(src, cnt, d.n, mask);
  __syncthreads();
  rescore_group<long long>(P.Jq + d.off_mat, P.hq + d.off_vec, d.n, d.n_pad, mask, red, cnt, gridDim.y,
                           reinterpret_cast<long long*>(P.rs_acc) + 2 * b0 * gridDim.y, gridDim.y,
                           [&](int g, long long Eq) { init_energy_out(P, d, b0 + g, Eq); });
}

__global__ void k_init_energy_finish(DevPtrs P, int b0, int nb, int parts) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= nb) return;
  const long long b = (long long)b0 + x;
  init_energy_out(P, P.inst[b / P.R], b, rs_energy(reinterpret_cast<const long long*>(P.rs_acc) + 2 * b * parts, parts));
}

cudaError_t launch_init_energy(const DevPtrs& P, int inst0, int n_inst, int max_n, cudaStream_t s) {
  if (n_inst <= 0) return cudaSuccess;
  const int ng = (P.R + kRG - 1) / kRG;
  const int parts = rescore_parts(P, n_inst * ng, max_n, true);
  const long long b0 = (long long)inst0 * P.R, nb = (long long)n_inst * P.R;
  const size_t sm = rescore_smem(P.NP, 8);
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_init_energy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_init_energy<<<dim3(n_inst * ng, parts), 256, sm, s>>>(P, inst0, ng);
  if (parts > 1) k_init_energy_finish<<<(int)((nb + 255) / 256), 256, 0, s>>>(P, (int)b0, (int)nb, parts);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- every instance's merged list
// Block (inst, group) for the states group * kRG ... of the first min(k, count of inst) of the
// merged list: their bits into out[inst][r][Wmax] and their energies, rescored as above, into
// E[inst][r]. The row parts: the exact form's when every instance is rescored exactly (split
// modes, on the grid), else the FP64 form's.
__global__ void __launch_bounds__(256) k_topk_all(DevPtrs P, int k, int all_exact, uint64_t* out, double* E) {
  const int ng = (k + kRG - 1) / kRG;
  const int inst = blockIdx.x / ng, g0 = (blockIdx.x % ng) * kRG;
  const int cnt = min(kRG, min(k, P.mrg_count[inst]) - g0);
  if (cnt <= 0) return;
  const InstDesc d = P.inst[inst];
  const bool exact = P.mode != QIS_FP64 && !d.rounded;
  // this instance's parts: the grid's when every instance is exact, else its FP64 number
  const int parts = all_exact ? (int)gridDim.y : fp64_parts(d.n);
  if ((int)blockIdx.y >= parts) return;
  extern __shared__ __align__(16) unsigned char rsm[];
  long long* redq = reinterpret_cast<long long*>(rsm);
  double* redd = reinterpret_cast<double*>(rsm);
  uint16_t* mask = reinterpret_cast<uint16_t*>(redq + 9 * (kRG + 1));
  __shared__ const uint64_t* src[kRG];
  if (threadIdx.x < kRG) {
    const int ref = P.mrg_ref[inst * P.K1 + g0 + min((int)threadIdx.x, cnt - 1)];
    src[threadIdx.x] = P.lst_bits + (long long)ref * P.Wmax;
  }
  __syncthreads();
  if (blockIdx.y == 0)
    for (int x = threadIdx.x; x < cnt * P.Wmax; x += blockDim.x) {
      const int g = x / P.Wmax, w = x - g * P.Wmax;
      out[((long long)inst * k + g0 + g) * P.Wmax + w] = (w < d.W) ? src[g][w] : 0ull;
    }
  group_masks(src, cnt, d.n, mask);
  __syncthreads();
  const long long o = (long long)inst * k + g0;
  const int PS = gridDim.y;
  if (exact)
    rescore_group<long long>(P.Jq + d.off_mat, P.hq + d.off_vec, d.n, d.n_pad, mask, redq, cnt, parts,
                             reinterpret_cast<long long*>(P.rs_acc) + 2 * o * PS, PS,
                             [&](int g, long long Eq) { E[o + g] = (double)Eq * d.inv_scale; });
  else
    rescore_group<double>(P.J64 + d.off_mat, P.h64 + d.off_vec, d.n, d.n_pad, mask, redd, cnt, parts,
                          reinterpret_cast<double*>(P.rs_acc) + 2 * o * PS, PS,
                          [&](int g, double Ev) { E[o + g] = Ev; });
}

__global__ void k_topk_all_finish(DevPtrs P, int k, int all_exact, int PS, double* E) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int inst = x / k, r = x - inst * k;
  if (inst >= P.n_inst || r >= min(k, P.mrg_count[inst])) return;
  const InstDesc d = P.inst[inst];
  const int parts = all_exact ? PS : fp64_parts(d.n);
  if (parts == 1) return;   // written by the rescoring block itself
  if (P.mode != QIS_FP64 && !d.rounded)
    E[x] = (double)rs_energy(reinterpret_cast<const long long*>(P.rs_acc) + 2ll * x * PS, parts) * d.inv_scale;
  else
    E[x] = rs_energy(reinterpret_cast<const double*>(P.rs_acc) + 2ll * x * PS, parts);
}

cudaError_t launch_topk_all(const DevPtrs& P, int k, bool all_exact, int max_n, uint64_t* out, double* E,
                            cudaStream_t s) {
  if (k <= 0 || P.n_inst <= 0) return cudaSuccess;
  const int groups = P.n_inst * ((k + kRG - 1) / kRG);
  const int parts = rescore_parts(P, groups, max_n, all_exact);
  const long long nstates = (long long)P.n_inst * k;
  const size_t sm = rescore_smem(P.NP, 8);
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_topk_all, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_topk_all<<<dim3(groups, parts), 256, sm, s>>>(P, k, all_exact ? 1 : 0, out, E);
  if (parts > 1) k_topk_all_finish<<<(int)((nstates + 255) / 256), 256, 0, s>>>(P, k, all_exact ? 1 : 0, parts, E);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- imported lists
// Zobrist hash of the first `count` slots of search b's list (the bits were copied in by the
// host): the same key the merge and the dedup use for states generated on the device.
__global__ void k_hash_list(DevPtrs P, int b, int count) {
  const InstDesc d = P.inst[b / P.R];
  const long long base = (long long)b * P.K1;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
    const uint64_t* bits = P.lst_bits + (base + k) * P.Wmax;
    uint64_t h = 0;
    for (int i = 0; i < d.n; ++i)
      if ((bits[i >> 6] >> (i & 63)) & 1ull) h ^= P.zob[i];
    P.lst_hash[base + k] = h;
  }
}

cudaError_t launch_hash_list(const DevPtrs& P, int b, int count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_hash_list<<<(count + 127) / 128, 128, 0, s>>>(P, b, count);
  return cudaGetLastError();
}

}  // namespace qis
