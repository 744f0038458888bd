// qis_iter.cu -- one iteration of Alg. 3 for every search of every instance (lockstep).
//
// Per iteration:
//   k_pick        parent = first unused kept state in key order (Alg. 3), marked used
//   k_fields_*    local fields of the parent; a_i = -2 s_i f_i
//   k_bound       per-search filter threshold (see below)
//   k_scan*       all single and pair flips, dE_i = a_i, dE_ij = a_i + a_j + 4 s_i s_j J_ij;
//                 survivors (candidate indices) appended per search
//   k_merge       exact energies of the survivors, duplicate removal (Zobrist hash + full
//                 compare), new list = first K+1 of old list + survivors by (E, stamp)
//
// Why a threshold suffices: a candidate enters the list only if its energy is below the
// last kept energy T (Alg. 2, strict <), and a state that leaves the list never comes back
// because T never increases. Hence one iteration of the sequential Alg. 2 loop leaves the
// same list as keeping the K+1 smallest keys (E, stamp) of the old list and of the new,
// non-duplicate candidates with E < T. The filter may therefore also drop every candidate
// whose energy exceeds any upper bound U on the (K+1+count)-th smallest candidate energy
// (at most `count` candidates duplicate a kept state). U is the (K+1+count)-th smallest
// energy among the single and pair flips of the m sites with the lowest a_i, a subset of the
// candidates, so U is never below the true order statistic.
#include "qis_common.cuh"

namespace qis {

__device__ inline float fl32_up(double x) { return __double2float_ru(x); }

// ---------------------------------------------------------------- parent pick (Alg. 3)
__global__ void __launch_bounds__(32) k_pick(DevPtrs P) {
  const int b = blockIdx.x;
  const InstDesc d = P.inst[b / P.R];
  const long long base = (long long)b * P.K1;
  const int lane = threadIdx.x;
  int sel = -1;
  if (P.active[b]) {
    const int cnt = P.lst_count[b];
    for (int r0 = 0; r0 < cnt && sel < 0; r0 += 32) {
      const int r = r0 + lane;
      int slot = -1;
      bool unused = false;
      if (r < cnt) {
        slot = P.lst_ord[base + r];
        unused = !P.lst_used[base + slot];
      }
      const unsigned m = __ballot_sync(0xffffffffu, unused);
      if (m) sel = __shfl_sync(0xffffffffu, slot, __ffs(m) - 1);
    }
  }
  if (lane == 0) {
    P.iter_t[b] += 1;
    if (sel < 0) {
      P.active[b] = 0;
    } else {
      P.lst_used[base + sel] = 1;
      P.par_E[b] = P.lst_E[base + sel];
      P.par_hash[b] = P.lst_hash[base + sel];
      atomicAdd(P.cand, (unsigned long long)d.n * (d.n - 1) / 2);
      atomicAdd(P.cand + 1, (unsigned long long)d.n);
    }
  }
  if (sel >= 0) {
    for (int w = lane; w < d.W; w += 32) P.par_bits[(long long)b * P.Wmax + w] = P.lst_bits[(base + sel) * P.Wmax + w];
    if (P.mode != QIS_FP64) {
      const uint64_t* src = P.lst_bits + (base + sel) * P.Wmax;
      for (int k = lane; k < d.n_pad; k += 32) {
        float v = (k < d.n) ? (sigma_of(src, k) ? -1.f : 1.f) : 0.f;
        P.S16[(long long)b * P.NP + k] = __float2bfloat16_rn(v);
      }
    }
  }
}

cudaError_t launch_pick(const DevPtrs& P, cudaStream_t s) {
  k_pick<<<P.B, 32, 0, s>>>(P);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- fields (exact integers, SIMT)
// fq_i = hq_i + sum_k Jq_ik s_k in int64 (exact); aq_i = -2 s_i fq_i; a32_i = fl32(aq_i 2^-q).
constexpr int kFS = 8;  // searches per thread
__global__ void __launch_bounds__(128) k_fields_exact(DevPtrs P) {
  const int inst = blockIdx.y;
  const InstDesc d = P.inst[inst];
  if ((int)blockIdx.x * 128 >= d.n_pad) return;
  const int i = blockIdx.x * 128 + threadIdx.x;
  const int s0 = blockIdx.z * kFS;
  const int ns = min(kFS, P.R - s0);
  __shared__ uint64_t sb[kFS][kMaxN / 64];
  __shared__ int act[kFS];
  for (int e = threadIdx.x; e < kFS * d.W; e += blockDim.x) {
    const int s = e / d.W, w = e % d.W;
    sb[s][w] = (s < ns) ? P.par_bits[(long long)(d.first_search + s0 + s) * P.Wmax + w] : 0ull;
  }
  if (threadIdx.x < kFS) act[threadIdx.x] = (threadIdx.x < ns) ? P.active[d.first_search + s0 + threadIdx.x] : 0;
  __syncthreads();
  long long acc[kFS];
#pragma unroll
  for (int s = 0; s < kFS; ++s) acc[s] = 0;
  const long long* Jq = P.Jq + d.off_mat;
  for (int k = 0; k < d.n; ++k) {
    const long long v = Jq[(long long)k * d.n_pad + i];   // Jq_ki = Jq_ik
#pragma unroll
    for (int s = 0; s < kFS; ++s) acc[s] += ((sb[s][k >> 6] >> (k & 63)) & 1ull) ? -v : v;
  }
  for (int s = 0; s < ns; ++s) {
    if (!act[s]) continue;
    const int b = d.first_search + s0 + s;
    long long aq = 0;
    float a32 = 0.f;
    if (i < d.n) {
      const long long fq = acc[s] + P.hq[d.off_vec + i];
      aq = ((sb[s][i >> 6] >> (i & 63)) & 1ull) ? 2 * fq : -2 * fq;
      a32 = (float)ldexp((double)aq, -d.q);
    }
    P.aq[(long long)b * P.NP + i] = aq;
    P.a32[(long long)b * P.NP + i] = a32;
  }
}

cudaError_t launch_fields_exact(const DevPtrs& P, cudaStream_t s) {
  dim3 g(P.NP / 128, P.n_inst, (P.R + kFS - 1) / kFS);
  k_fields_exact<<<g, 128, 0, s>>>(P);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- fields (FP64 plain form)
// f_i = (sum_{j != i} s_j J_ij, j ascending from +0.0) + h_i; a_i = -2 s_i f_i. The order of
// the additions is fixed so the result is reproducible bit for bit.
__global__ void __launch_bounds__(128) k_fields_fp64(DevPtrs P) {
  const int inst = blockIdx.y;
  const InstDesc d = P.inst[inst];
  if ((int)blockIdx.x * 128 >= d.n_pad) return;
  const int i = blockIdx.x * 128 + threadIdx.x;
  const int s0 = blockIdx.z * kFS;
  const int ns = min(kFS, P.R - s0);
  __shared__ uint64_t sb[kFS][kMaxN / 64];
  __shared__ int act[kFS];
  for (int e = threadIdx.x; e < kFS * d.W; e += blockDim.x) {
    const int s = e / d.W, w = e % d.W;
    sb[s][w] = (s < ns) ? P.par_bits[(long long)(d.first_search + s0 + s) * P.Wmax + w] : 0ull;
  }
  if (threadIdx.x < kFS) act[threadIdx.x] = (threadIdx.x < ns) ? P.active[d.first_search + s0 + threadIdx.x] : 0;
  __syncthreads();
  double acc[kFS];
#pragma unroll
  for (int s = 0; s < kFS; ++s) acc[s] = 0.0;
  const double* J = P.J64 + d.off_mat;
  const int ic = min(i, d.n_pad - 1);
  for (int j = 0; j < d.n; ++j) {
    if (j == i) continue;
    const double v = J[(long long)j * d.n_pad + ic];      // J_ji = J_ij
#pragma unroll
    for (int s = 0; s < kFS; ++s) acc[s] = __dadd_rn(acc[s], ((sb[s][j >> 6] >> (j & 63)) & 1ull) ? -v : v);
  }
  for (int s = 0; s < ns; ++s) {
    if (!act[s]) continue;
    const int b = d.first_search + s0 + s;
    double a = 0.0;
    if (i < d.n) {
      const double f = __dadd_rn(acc[s], P.h64[d.off_vec + i]);
      a = ((sb[s][i >> 6] >> (i & 63)) & 1ull) ? 2.0 * f : -2.0 * f;
    }
    P.a64[(long long)b * P.NP + i] = a;
  }
}

cudaError_t launch_fields_fp64(const DevPtrs& P, cudaStream_t s) {
  dim3 g(P.NP / 128, P.n_inst, (P.R + kFS - 1) / kFS);
  k_fields_fp64<<<g, 128, 0, s>>>(P);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- block bitonic sort
template <typename K>
__device__ void bitonic_sort(K* key, uint32_t* val, int n2) {
  for (int k = 2; k <= n2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < n2; t += blockDim.x) {
        const int u = t ^ j;
        if (u > t) {
          const K a = key[t], c = key[u];
          const uint32_t va = val[t], vc = val[u];
          const bool gt = (a > c) || (a == c && va > vc);
          const bool up = (t & k) == 0;
          if (gt == up) {
            key[t] = c; key[u] = a;
            val[t] = vc; val[u] = va;
          }
        }
      }
      __syncthreads();
    }
  }
}

__device__ inline int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// candidate energy change in the scan's arithmetic
__device__ inline float dE32(float ai, float aj, float j4, int flip) {
  return (ai + aj) + __int_as_float(__float_as_int(j4) ^ (flip << 31));
}
__device__ inline double dE64(double ai, double aj, double j, int flip) {
  // (a_i + a_j) + 4 s_i s_j J_ij; the product 4 s_i s_j J_ij is exact
  return __dadd_rn(__dadd_rn(ai, aj), flip ? -4.0 * j : 4.0 * j);
}

// ---------------------------------------------------------------- per-search bound
constexpr int kMaxSub = 3968;  // subset values; keeps the padded sort within kMaxN
// Dynamic shared memory: vals (kMaxN floats/doubles as u64 keys) + idx.
__global__ void __launch_bounds__(256) k_bound(DevPtrs P) {
  const int b = blockIdx.x;
  const InstDesc d = P.inst[b / P.R];
  const long long base = (long long)b * P.K1;
  if (!P.active[b]) {
    if (threadIdx.x == 0) {
      P.surv_cnt[b] = 0;
      P.thr32[b] = -INFINITY;
      P.thrE[b] = -INFINITY;
      P.capE[b] = -INFINITY;
    }
    return;
  }
  extern __shared__ unsigned char smem[];
  unsigned long long* key = reinterpret_cast<unsigned long long*>(smem);        // [max(npow2, subpow2)]
  uint32_t* idx = reinterpret_cast<uint32_t*>(key + kMaxN);                      // [same]
  __shared__ float s_amax;
  __shared__ uint64_t pb[kMaxN / 64];
  const int n = d.n;
  const bool fp64 = P.mode == QIS_FP64;
  const int cnt = P.lst_count[b];
  const double T = (cnt == P.K1) ? P.lst_E[base + P.lst_ord[base + P.K1 - 1]] : INFINITY;
  const double Ep = P.par_E[b];
  const long long C = (long long)n * (n + 1) / 2;
  const int k = P.K1 + cnt;
  for (int w = threadIdx.x; w < d.W; w += blockDim.x) pb[w] = P.par_bits[(long long)b * P.Wmax + w];
  if (threadIdx.x == 0) s_amax = 0.f;
  __syncthreads();
  const float* a32 = P.a32 + (long long)b * P.NP;
  const double* a64 = P.a64 + (long long)b * P.NP;
  if (!fp64) {
    float m = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmaxf(m, fabsf(a32[i]));
    atomicMax(reinterpret_cast<int*>(&s_amax), __float_as_int(m));   // non-negative floats order as ints
  }
  double U = INFINITY;
  if (C > k) {
    // m lowest a_i: sort (a_i, i) ascending
    const int n2 = next_pow2(n);
    for (int i = threadIdx.x; i < n2; i += blockDim.x) {
      key[i] = (i < n) ? dkey(fp64 ? a64[i] : (double)a32[i]) : ~0ull;
      idx[i] = i;
    }
    __syncthreads();
    bitonic_sort(key, idx, n2);
    int want = min(4 * k, kMaxSub);
    int m = 1;
    while (m < n && m + m * (m - 1) / 2 < want) ++m;
    const int M = m + m * (m - 1) / 2;
    // copy the m sites out of idx before key/idx are reused
    __shared__ int sites[128];
    const int msafe = min(m, 128);
    for (int x = threadIdx.x; x < msafe; x += blockDim.x) sites[x] = idx[x];
    __syncthreads();
    const int mm = msafe;
    const int MM = mm + mm * (mm - 1) / 2;
    const int M2 = next_pow2(MM);
    for (int t = threadIdx.x; t < M2; t += blockDim.x) {
      unsigned long long kk = ~0ull;
      if (t < MM) {
        int i, j;
        if (t < mm) {
          i = sites[t]; j = -1;
        } else {
          // pair number r among the mm sites: x < y lexicographic
          int r = t - mm, x = 0;
          while (r >= mm - 1 - x) { r -= mm - 1 - x; ++x; }
          i = sites[x]; j = sites[x + 1 + r];
          if (i > j) { int tmp = i; i = j; j = tmp; }
        }
        if (fp64) {
          double de;
          if (j < 0) de = a64[i];
          else de = dE64(a64[i], a64[j], P.J64[d.off_mat + (long long)i * d.n_pad + j],
                         sigma_of(pb, i) ^ sigma_of(pb, j));
          kk = dkey(__dadd_rn(Ep, de));
        } else {
          float de;
          if (j < 0) de = a32[i];
          else de = dE32(a32[i], a32[j], P.J4[d.off_mat + (long long)i * d.n_pad + j], sigma_of(pb, i) ^ sigma_of(pb, j));
          kk = dkey((double)de);
        }
      }
      key[t] = kk;
      idx[t] = t;
    }
    __syncthreads();
    bitonic_sort(key, idx, M2);
    (void)M;
    if (k - 1 < MM) {
      unsigned long long u = key[k - 1];
      u = (u & 0x8000000000000000ull) ? (u & 0x7fffffffffffffffull) : ~u;
      U = __longlong_as_double((long long)u);
    }
  }
  __syncthreads();   // s_amax complete
  if (threadIdx.x == 0) {
    P.surv_cnt[b] = 0;
    if (fp64) {
      P.thrE[b] = T;
      P.capE[b] = U;
    } else {
      // |dE~ - dE| <= delta: a32 and J4 are fl32 of exact values, plus two fl32 additions
      const double delta = ldexp(2.0 * (double)s_amax + (double)d.j4max, -21);
      const double t1 = (T == INFINITY) ? INFINITY : (T - Ep) + delta;   // T - Ep is exact
      const double t2 = U + 2.0 * delta;
      P.thr32[b] = fl32_up(fmin(t1, t2));
    }
  }
}

cudaError_t launch_bound(const DevPtrs& P, cudaStream_t s) {
  const size_t sm = (size_t)kMaxN * (8 + 4);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_bound, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = true;
  }
  k_bound<<<P.B, 256, sm, s>>>(P);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- candidate scan (FP32 filter)
// One block per 64 x 64 tile (bi <= bj) of one instance; the tile of fl32(4 J) is loaded once
// and reused for all R searches of the instance. Thread (ty, tx) owns rows 4ty..4ty+3 and
// columns 4tx..4tx+3 of the tile. Pair (i, j), i < j, survives if dE~ <= thr; on a diagonal
// tile the i == j positions carry the single flips.
__global__ void __launch_bounds__(256) k_scan32(DevPtrs P, const int4* work) {
  const int4 w = work[blockIdx.x];
  const InstDesc d = P.inst[w.x];
  const int n = d.n, np = d.n_pad;
  const int i0 = w.y * kTile, j0 = w.z * kTile;
  const bool diag = w.y == w.z;
  __shared__ float Jt[kTile][kTile + 1];
  __shared__ float ar_s[kTile], ac_s[kTile];
  const float* J4 = P.J4 + d.off_mat;
  for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
    const int r = e >> 6, c = e & 63;
    Jt[r][c] = J4[(long long)(i0 + r) * np + j0 + c];
  }
  __syncthreads();
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  float jr[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) jr[r][c] = Jt[ty * 4 + r][tx * 4 + c];
  for (int s = 0; s < P.R; ++s) {
    const int b = d.first_search + s;
    __syncthreads();
    if (!P.active[b]) continue;
    const float* a = P.a32 + (long long)b * P.NP;
    if (threadIdx.x < kTile) ar_s[threadIdx.x] = a[i0 + threadIdx.x];
    else if (threadIdx.x < 2 * kTile) ac_s[threadIdx.x - kTile] = a[j0 + threadIdx.x - kTile];
    __syncthreads();
    const float thr = P.thr32[b];
    const uint64_t wi = P.par_bits[(long long)b * P.Wmax + w.y];
    const uint64_t wj = P.par_bits[(long long)b * P.Wmax + w.z];
    const unsigned rs = (unsigned)(wi >> (ty * 4)) & 15u, cs = (unsigned)(wj >> (tx * 4)) & 15u;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = i0 + ty * 4 + r;
      const float ai = ar_s[ty * 4 + r];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int j = j0 + tx * 4 + c;
        bool ok;
        uint32_t cid;
        if (diag && i >= j) {
          ok = (i == j) && (i < n) && (ai <= thr);
          cid = (uint32_t)i;
        } else {
          const int flip = ((rs >> r) ^ (cs >> c)) & 1;
          const float y = dE32(ai, ac_s[tx * 4 + c], jr[r][c], flip);
          ok = (j < n) && (y <= thr);
          cid = pair_index(n, i, j);
        }
        if (ok) {
          const int slot = atomicAdd(P.surv_cnt + b, 1);
          if (slot < P.cap) P.surv[(long long)b * P.cap + slot] = cid;
        }
      }
    }
  }
}

// FP64 plain form: E' = E_p + dE exactly as defined; survivors have E' < T and E' <= cap.
__global__ void __launch_bounds__(256) k_scan64(DevPtrs P, const int4* work) {
  const int4 w = work[blockIdx.x];
  const InstDesc d = P.inst[w.x];
  const int n = d.n, np = d.n_pad;
  const int i0 = w.y * kTile, j0 = w.z * kTile;
  const bool diag = w.y == w.z;
  __shared__ double Jt[kTile][kTile + 1];
  __shared__ double ar_s[kTile], ac_s[kTile];
  const double* J = P.J64 + d.off_mat;
  for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
    const int r = e >> 6, c = e & 63;
    Jt[r][c] = J[(long long)(i0 + r) * np + j0 + c];
  }
  __syncthreads();
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  for (int s = 0; s < P.R; ++s) {
    const int b = d.first_search + s;
    __syncthreads();
    if (!P.active[b]) continue;
    const double* a = P.a64 + (long long)b * P.NP;
    if (threadIdx.x < kTile) ar_s[threadIdx.x] = a[i0 + threadIdx.x];
    else if (threadIdx.x < 2 * kTile) ac_s[threadIdx.x - kTile] = a[j0 + threadIdx.x - kTile];
    __syncthreads();
    const double T = P.thrE[b], cap = P.capE[b], Ep = P.par_E[b];
    const uint64_t wi = P.par_bits[(long long)b * P.Wmax + w.y];
    const uint64_t wj = P.par_bits[(long long)b * P.Wmax + w.z];
    const unsigned rs = (unsigned)(wi >> (ty * 4)) & 15u, cs = (unsigned)(wj >> (tx * 4)) & 15u;
    for (int r = 0; r < 4; ++r) {
      const int i = i0 + ty * 4 + r;
      const double ai = ar_s[ty * 4 + r];
      for (int c = 0; c < 4; ++c) {
        const int j = j0 + tx * 4 + c;
        bool ok;
        uint32_t cid;
        if (diag && i >= j) {
          const double e = __dadd_rn(Ep, ai);
          ok = (i == j) && (i < n) && (e < T) && (e <= cap);
          cid = (uint32_t)i;
        } else {
          const int flip = ((rs >> r) ^ (cs >> c)) & 1;
          const double e = __dadd_rn(Ep, dE64(ai, ac_s[tx * 4 + c], Jt[ty * 4 + r][tx * 4 + c], flip));
          ok = (j < n) && (e < T) && (e <= cap);
          cid = pair_index(n, i, j);
        }
        if (ok) {
          const int slot = atomicAdd(P.surv_cnt + b, 1);
          if (slot < P.cap) P.surv[(long long)b * P.cap + slot] = cid;
        }
      }
    }
  }
}

cudaError_t launch_scan(const DevPtrs& P, const int4* work, int n_work, cudaStream_t s) {
  if (n_work <= 0) return cudaSuccess;
  if (P.mode == QIS_FP64) k_scan64<<<n_work, 256, 0, s>>>(P, work);
  else k_scan32<<<n_work, 256, 0, s>>>(P, work);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- exact merge (Alg. 2)
// Shared layout (dynamic): old list [K1] {E, hash, slot}, survivors [P2] {key, cand},
// rank/slot scratch [K1].
__global__ void __launch_bounds__(256) k_merge(DevPtrs P) {
  const int b = blockIdx.x;
  if (!P.active[b]) return;
  const InstDesc d = P.inst[b / P.R];
  const int n = d.n, W = d.W, K1 = P.K1;
  const long long base = (long long)b * K1;
  const int S = P.surv_cnt[b];
  if (S > P.cap) {
    if (threadIdx.x == 0) atomicOr(P.status, kStatCapacity);
    return;
  }
  extern __shared__ unsigned char smem[];
  const int P2 = next_pow2(max(S, 1));
  double* oE = reinterpret_cast<double*>(smem);                 // [K1]
  uint64_t* oH = reinterpret_cast<uint64_t*>(oE + K1);          // [K1]
  unsigned long long* sk = reinterpret_cast<unsigned long long*>(oH + K1);   // [P2]
  uint32_t* sc = reinterpret_cast<uint32_t*>(sk + P2);          // [P2]
  int* oslot = reinterpret_cast<int*>(sc + P2);                 // [K1]
  int* occ = oslot + K1;                                        // [K1]
  int* freel = occ + K1;                                        // [K1]
  __shared__ uint64_t pb[kMaxN / 64];
  __shared__ int s_nvalid, s_nfree;
  const int cnt = P.lst_count[b];
  const double T = (cnt == K1) ? P.lst_E[base + P.lst_ord[base + K1 - 1]] : INFINITY;
  const double Ep = P.par_E[b];
  const uint64_t ph = P.par_hash[b];
  const bool fp64 = P.mode == QIS_FP64;
  for (int w = threadIdx.x; w < W; w += blockDim.x) pb[w] = P.par_bits[(long long)b * P.Wmax + w];
  for (int r = threadIdx.x; r < cnt; r += blockDim.x) {
    const int slot = P.lst_ord[base + r];
    oslot[r] = slot;
    oE[r] = P.lst_E[base + slot];
    oH[r] = P.lst_hash[base + slot];
  }
  for (int k = threadIdx.x; k < K1; k += blockDim.x) occ[k] = 0;
  if (threadIdx.x == 0) s_nvalid = 0;
  __syncthreads();
  const long long Epq = fp64 ? 0 : __double2ll_rn(ldexp(Ep, d.q));
  const long long Tq = (fp64 || T == INFINITY) ? LLONG_MAX : __double2ll_rn(ldexp(T, d.q));
  for (int t = threadIdx.x; t < P2; t += blockDim.x) {
    unsigned long long kk = ~0ull;
    uint32_t c = 0xffffffffu;
    if (t < S) {
      c = P.surv[(long long)b * P.cap + t];
      int i, j;
      decode_candidate(n, c, i, j);
      const int si = sigma_of(pb, i), sj = (j >= 0) ? sigma_of(pb, j) : 0;
      double e;
      bool keep;
      if (fp64) {
        const double* a = P.a64 + (long long)b * P.NP;
        const double de = (j < 0) ? a[i] : dE64(a[i], a[j], P.J64[d.off_mat + (long long)i * d.n_pad + j], si ^ sj);
        e = __dadd_rn(Ep, de);
        keep = e < T;
      } else {
        const long long* aq = P.aq + (long long)b * P.NP;
        long long de = aq[i];
        if (j >= 0) {
          const long long jq = P.Jq[d.off_mat + (long long)i * d.n_pad + j];
          de += aq[j] + ((si ^ sj) ? -4 * jq : 4 * jq);
        }
        const long long eq = Epq + de;
        keep = eq < Tq;
        e = ldexp((double)eq, -d.q);
      }
      if (keep) {
        const uint64_t hsh = ph ^ P.zob[i] ^ ((j >= 0) ? P.zob[j] : 0ull);
        for (int r = 0; r < cnt && keep; ++r) {
          if (oH[r] != hsh) continue;
          const uint64_t* sbits = P.lst_bits + (base + oslot[r]) * P.Wmax;
          bool same = true;
          for (int x = 0; x < W && same; ++x) {
            uint64_t m = 0;
            if ((i >> 6) == x) m ^= 1ull << (i & 63);
            if (j >= 0 && (j >> 6) == x) m ^= 1ull << (j & 63);
            same = sbits[x] == (pb[x] ^ m);
          }
          if (same) keep = false;   // duplicate of a kept state (Alg. 2 binary search hit)
        }
      }
      if (keep) {
        kk = dkey(e);
        atomicAdd(&s_nvalid, 1);
      } else {
        c = 0xffffffffu;
      }
    }
    sk[t] = kk;
    sc[t] = c;
  }
  __syncthreads();
  bitonic_sort(sk, sc, P2);
  const int nv = s_nvalid;
  // ranks: old entry o -> o + #(new with E < E_o); new entry p -> p + #(old with E <= E_p)
  // (new stamps exceed every old stamp, and among new entries c orders the stamps)
  for (int o = threadIdx.x; o < cnt; o += blockDim.x) {
    const unsigned long long ko = dkey(oE[o]);
    int lo = 0, hi = nv;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (sk[mid] < ko) lo = mid + 1; else hi = mid;
    }
    const int rank = o + lo;
    if (rank < K1) occ[oslot[o]] = 1 + rank;   // kept: remember rank + 1
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int nf = 0;
    for (int k = 0; k < K1; ++k)
      if (!occ[k]) freel[nf++] = k;
    s_nfree = nf;
  }
  __syncthreads();
  const int t_now = P.iter_t[b];
  for (int p = threadIdx.x; p < nv; p += blockDim.x) {
    const unsigned long long kp = sk[p];
    int lo = 0, hi = cnt;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (dkey(oE[mid]) <= kp) lo = mid + 1; else hi = mid;
    }
    const int rank = p + lo;
    if (rank >= K1) continue;
    const int slot = freel[p];   // new entries kept are exactly the first ones in sorted order
    const uint32_t c = sc[p];
    int i, j;
    decode_candidate(n, c, i, j);
    uint64_t* dst = P.lst_bits + (base + slot) * P.Wmax;
    for (int x = 0; x < W; ++x) {
      uint64_t m = 0;
      if ((i >> 6) == x) m ^= 1ull << (i & 63);
      if (j >= 0 && (j >> 6) == x) m ^= 1ull << (j & 63);
      dst[x] = pb[x] ^ m;
    }
    unsigned long long u = kp;
    u = (u & 0x8000000000000000ull) ? (u & 0x7fffffffffffffffull) : ~u;
    P.lst_E[base + slot] = __longlong_as_double((long long)u);
    P.lst_stamp[base + slot] = ((uint64_t)t_now << 32) | c;
    P.lst_hash[base + slot] = ph ^ P.zob[i] ^ ((j >= 0) ? P.zob[j] : 0ull);
    P.lst_used[base + slot] = 0;
    P.lst_ord[base + rank] = slot;
  }
  for (int o = threadIdx.x; o < cnt; o += blockDim.x) {
    const int slot = oslot[o];
    if (occ[slot]) P.lst_ord[base + occ[slot] - 1] = slot;
  }
  if (threadIdx.x == 0) P.lst_count[b] = min(K1, cnt + nv);
}

size_t merge_smem(int K1, int cap) {
  const int P2 = [](int x) { int p = 1; while (p < x) p <<= 1; return p; }(cap);
  return (size_t)K1 * (8 + 8) + (size_t)P2 * (8 + 4) + (size_t)K1 * 4 * 3;
}

cudaError_t launch_merge(const DevPtrs& P, cudaStream_t s) {
  const size_t sm = merge_smem(P.K1, P.cap);
  static size_t attr = 0;
  if (attr < sm) {
    cudaFuncSetAttribute(k_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = sm;
  }
  k_merge<<<P.B, 256, sm, s>>>(P);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- Alg. 4 merge
// One block per instance. Search 0's list seeds the merged list; the lists of searches
// 1..R-1 are merged in turn. A state already present is skipped (its first occurrence
// wins); the rest are ranked by (E, search, position) and the first K+1 kept.
__global__ void __launch_bounds__(256) k_final_merge(DevPtrs P) {
  const int inst = blockIdx.x;
  const InstDesc d = P.inst[inst];
  const int K1 = P.K1, W = d.W;
  extern __shared__ unsigned char smem[];
  // 8-byte arrays first, then 4-byte arrays (keeps every array aligned for any K1)
  double* aE = reinterpret_cast<double*>(smem);                               // accumulated list
  unsigned long long* aS = reinterpret_cast<unsigned long long*>(aE + K1);    // src
  uint64_t* aH = reinterpret_cast<uint64_t*>(aS + K1);
  double* nE = reinterpret_cast<double*>(aH + K1);                            // incoming list
  unsigned long long* nS = reinterpret_cast<unsigned long long*>(nE + K1);
  uint64_t* nH = reinterpret_cast<uint64_t*>(nS + K1);
  double* tE = reinterpret_cast<double*>(nH + K1);                            // staging
  unsigned long long* tS = reinterpret_cast<unsigned long long*>(tE + K1);
  uint64_t* tH = reinterpret_cast<uint64_t*>(tS + K1);
  int* aR = reinterpret_cast<int*>(tH + K1);                                  // ref = b*K1 + slot
  int* nR = aR + K1;
  int* tR = nR + K1;
  int* nDup = tR + K1;
  int* nPos = nDup + K1;
  __shared__ int s_acnt, s_ncnt;
  for (int r = 0; r < P.R; ++r) {
    const int b = d.first_search + r;
    const long long base = (long long)b * K1;
    const int cnt = P.lst_count[b];
    for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
      const int slot = P.lst_ord[base + p];
      nE[p] = P.lst_E[base + slot];
      nH[p] = P.lst_hash[base + slot];
      nR[p] = (int)(base + slot);
      nS[p] = ((unsigned long long)r << 32) | (unsigned)p;
    }
    if (r == 0) {
      __syncthreads();
      for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
        aE[p] = nE[p]; aH[p] = nH[p]; aR[p] = nR[p]; aS[p] = nS[p];
      }
      if (threadIdx.x == 0) s_acnt = cnt;
      __syncthreads();
      continue;
    }
    __syncthreads();
    const int acnt = s_acnt;
    for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
      int dup = 0;
      for (int a = 0; a < acnt && !dup; ++a) {
        if (aH[a] != nH[p]) continue;
        const uint64_t* x = P.lst_bits + (long long)aR[a] * P.Wmax;
        const uint64_t* y = P.lst_bits + (long long)nR[p] * P.Wmax;
        bool same = true;
        for (int w = 0; w < W && same; ++w) same = x[w] == y[w];
        dup = same;
      }
      nDup[p] = dup;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int m = 0;
      for (int p = 0; p < cnt; ++p) {
        nPos[p] = nDup[p] ? -1 : m;
        if (!nDup[p]) ++m;
      }
      s_ncnt = m;
    }
    __syncthreads();
    const int m = s_ncnt;
    // compacted incoming entries go to the tail arrays' "new" view via nPos
    for (int a = threadIdx.x; a < acnt; a += blockDim.x) {
      // # incoming non-duplicates with E < aE[a]
      int less = 0;
      for (int p = 0; p < cnt; ++p)
        if (nPos[p] >= 0 && nE[p] < aE[a]) ++less;
      const int rank = a + less;
      if (rank < K1) { tE[rank] = aE[a]; tS[rank] = aS[a]; tH[rank] = aH[a]; tR[rank] = aR[a]; }
    }
    for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
      if (nPos[p] < 0) continue;
      int le = 0;
      for (int a = 0; a < acnt; ++a)
        if (aE[a] <= nE[p]) ++le;
      const int rank = nPos[p] + le;
      if (rank < K1) { tE[rank] = nE[p]; tS[rank] = nS[p]; tH[rank] = nH[p]; tR[rank] = nR[p]; }
    }
    __syncthreads();
    const int ncnt = min(K1, acnt + m);
    for (int a = threadIdx.x; a < ncnt; a += blockDim.x) {
      aE[a] = tE[a]; aS[a] = tS[a]; aH[a] = tH[a]; aR[a] = tR[a];
    }
    if (threadIdx.x == 0) s_acnt = ncnt;
    __syncthreads();
  }
  const int acnt = s_acnt;
  for (int a = threadIdx.x; a < K1; a += blockDim.x) {
    P.mrg_ref[inst * K1 + a] = (a < acnt) ? aR[a] : -1;
    P.mrg_src[inst * K1 + a] = (a < acnt) ? aS[a] : ~0ull;
  }
  if (threadIdx.x == 0) P.mrg_count[inst] = acnt;
}

size_t final_merge_smem(int K1) { return (size_t)K1 * (9 * 8 + 5 * 4); }

cudaError_t launch_final_merge(const DevPtrs& P, cudaStream_t s) {
  const size_t sm = final_merge_smem(P.K1);
  static size_t attr = 0;
  if (attr < sm) {
    cudaFuncSetAttribute(k_final_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = sm;
  }
  k_final_merge<<<P.n_inst, 256, sm, s>>>(P);
  return cudaGetLastError();
}

}  // namespace qis
