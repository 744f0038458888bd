// qis_iter.cu -- one iteration of Alg. 3 for every search of every instance (lockstep).
//
// Per iteration:
//   k_pick        parent = first unused kept state in key order (Alg. 3), marked used
//   k_fields_*    local fields of the parent (by update from its generator's exact fields,
//                 else the tensor-core GEMM); a_i = -2 s_i f_i (energy change of flip i)
//   k_bound       per-search filter threshold; single flips dE_i = a_i tested here; the
//                 candidate indices of the kept states one or two flips from the parent
//   k_scan_*      pair flips dE_ij = a_i + a_j + 4 s_i s_j J_ij; survivors appended
//   k_merge       exact energies of the survivors, duplicate removal (by candidate index),
//                 new list = first K+1 of old list + survivors by (E, stamp)
//
// Why a threshold suffices: a candidate enters the list only if its energy is below the
// last kept energy T (Alg. 2, strict <), and a state that leaves the list never comes back
// because T never increases. Hence one iteration of the sequential Alg. 2 loop leaves the
// same list as keeping the K+1 smallest keys (E, stamp) of the old list and of the new,
// non-duplicate candidates with E < T. The filter may therefore also drop every candidate
// whose energy exceeds any upper bound U on the (K+1+count)-th smallest candidate energy
// (at most `count` candidates duplicate a kept state). U is taken as the (K+1+count)-th
// smallest energy among the single and pair flips of a few sites with the lowest a_i, a
// subset of the candidates, so it never lies below the true order statistic.
#include "qis_block.cuh"

namespace qis {


// ---------------------------------------------------------------- parent pick (Alg. 3)
// One warp per search, four searches per block (more searches resident than with one-warp
// blocks: the per-search chain of dependent loads is what takes the time).
__global__ void __launch_bounds__(128) k_pick(DevPtrs P) {
  const int b = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (b >= P.B) return;   // warp-uniform
  const InstDesc d = P.inst[b / P.R];
  const long long base = (long long)b * P.K1;
  const int lane = threadIdx.x & 31;
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
    const int r = b % P.R;   // clear the tile's full-fields flag (set again by k_fields_inc)
    if (P.gemm_nt > 0 && r % P.gemm_nt == 0)
      P.full_tile[(b / P.R) * ((P.R + P.gemm_nt - 1) / P.gemm_nt) + r / P.gemm_nt] = 0;
    if (sel < 0) {
      P.active[b] = 0;
    } else {
      P.lst_used[base + sel] = 1;
      if (P.mode == QIS_FP64) P.par_E[b] = P.lst_E[base + sel];   // split modes: par_q
      if (P.mode != QIS_FP64) P.par_q[b] = P.lst_q[base + sel];
      P.par_hash[b] = P.lst_hash[base + sel];
      P.par_stamp[b] = P.lst_stamp[base + sel];
      P.nprod[b] += 1;   // n(n-1)/2 pair and n single candidates, counted on query
    }
  }
  if (sel >= 0) {
    int down = 0;   // spins -1 of the parent (sigma = 1)
    for (int w = lane; w < d.W; w += 32) {
      const uint64_t x = P.lst_bits[(base + sel) * P.Wmax + w];
      P.par_bits[(long long)b * P.Wmax + w] = x;
      down += __popcll(x);
    }
    for (int o = 16; o > 0; o >>= 1) down += __shfl_xor_sync(0xffffffffu, down, o);
    if (lane == 0) {   // pair candidates of this parent for the flip set
      const unsigned long long nn = (unsigned long long)d.n;
      P.npair[b] += (P.flips == QIS_FLIPS_SINGLE)     ? 0ull
                    : (P.flips == QIS_FLIPS_EXCHANGE) ? (unsigned long long)down * (nn - (unsigned long long)down)
                                                      : nn * (nn - 1) / 2;
    }
    if (P.mode != QIS_FP64) {
      const uint64_t* src = P.lst_bits + (base + sel) * P.Wmax;
      __half* dst = P.S16 + (long long)(b / P.R) * P.s16_stride;
      const int r = b % P.R;
      for (int k = lane; k < d.n_pad; k += 32) {
        float v = (k < d.n) ? (sigma_of(src, k) ? -1.f : 1.f) : 0.f;
        dst[s16_offset(r, k, P.gemm_nt, P.NP)] = __float2half_rn(v);
      }
    }
  }
}

cudaError_t launch_pick(const DevPtrs& P, cudaStream_t s) {
  k_pick<<<(P.B + 3) / 4, 128, 0, s>>>(P);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- fields (exact integers, SIMT)
// fq_i = hq_i + sum_k Jq_ik s_k in int64 (exact); aq_i = -2 s_i fq_i;
// as32_i = {fl32(aq_i 2^-q), s_i}.
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
    float a32 = 0.f, s32 = 0.f;
    if (i < d.n) {
      const int sg = (int)((sb[s][i >> 6] >> (i & 63)) & 1ull);
      const long long fq = acc[s] + P.hq[d.off_vec + i];
      aq = sg ? 2 * fq : -2 * fq;
      a32 = (float)ldexp((double)aq, -d.q);
      s32 = sg ? -1.f : 1.f;
    }
    aq_of(P, b, P.iter_t[b])[i] = aq;
    P.as32[(long long)b * P.NP + i] = make_float2(a32, s32);
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
  for (int j = 0; j < d.n; ++j) {
    if (j == i) continue;
    const double v = J[(long long)j * d.n_pad + i];      // J_ji = J_ij
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

// ---------------------------------------------------------------- fields by update (split modes)
// A kept state x entered the list at iteration tg (its stamp) as a flip of site i, or of sites
// i and j, of that iteration's parent g, whose exact fields are in the aq ring. With s_g the
// spins of g (s_x with i, j flipped back) the exact integer fields of x follow in O(n):
//   fq_k(x) = fq_k(g) - 2 s_g,i Jq_ki - 2 s_g,j Jq_kj        (Jq_kk = 0)
// from fq_k(g) = -s_g,k aq_k(g) / 2, and aq_k(x) = -2 s_x,k fq_k(x). The result equals the
// field GEMM's bit for bit (both exact). A parent without a ring entry of its generator (the
// initial state, an imported list, a generator more than ring_n iterations back) marks its
// tensor-core tile, and the GEMM computes that tile in full.
__global__ void __launch_bounds__(256, 8) k_fields_inc(DevPtrs P) {
  const int b = blockIdx.x;
  // every load that depends only on b, issued together
  const int act = P.active[b], t = P.iter_t[b], t0 = P.ring_t0[b];
  const uint64_t st = P.par_stamp[b];
  const InstDesc d = P.inst[b / P.R];
  __shared__ uint64_t xb[kMaxN / 64];
  for (int w = threadIdx.x; w < P.Wmax; w += blockDim.x) xb[w] = P.par_bits[(long long)b * P.Wmax + w];
  __syncthreads();
  if (!act) return;
  const int tg = (int)(st >> 32);
  if (!(tg >= 1 && tg > t0 && tg < t && t - tg < P.ring_n)) {
    if (threadIdx.x == 0) {
      const int r = b % P.R;
      P.full_tile[(b / P.R) * ((P.R + P.gemm_nt - 1) / P.gemm_nt) + r / P.gemm_nt] = 1;
    }
    return;
  }
  int i, j;
  decode_candidate(d.n, (uint32_t)st, i, j);
  // 2 s_g at the flipped sites: s_g = -s_x there, s_x = -1 where sigma = 1
  const long long gi = sigma_of(xb, i) ? 2 : -2;
  const long long gj = (j >= 0) ? (sigma_of(xb, j) ? 2 : -2) : 0;
  const long long* __restrict__ ag = aq_of(P, b, tg);
  long long* __restrict__ ax = aq_of(P, b, t);
  float2* __restrict__ as = P.as32 + (long long)b * P.NP;
  const long long* __restrict__ Ji = P.Jq + d.off_mat + (long long)i * d.n_pad;   // row i = column i
  const long long* __restrict__ Jj = P.Jq + d.off_mat + (long long)max(j, 0) * d.n_pad;
  const float scale_q = (float)d.inv_scale;
  constexpr int U = 4;   // sites per thread and pass, their loads issued together
  for (int k0 = 0; k0 < d.n_pad; k0 += U * 256) {
    long long vg[U], vi[U], vj[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + u * 256 + threadIdx.x;
      vg[u] = vi[u] = vj[u] = 0;
      if (k < d.n) {
        vg[u] = ag[k];
        vi[u] = Ji[k];
        if (j >= 0) vj[u] = Jj[k];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + u * 256 + threadIdx.x;
      if (k >= d.n_pad) break;
      long long aq = 0;
      float2 a = make_float2(0.f, 0.f);
      if (k < d.n) {
        const int sx = sigma_of(xb, k);
        const int sg = sx ^ (k == i || k == j);
        const long long fg = sg ? vg[u] / 2 : -(vg[u] / 2);   // aq = -2 s f, s = -1 where sigma = 1
        const long long fx = fg - gi * vi[u] - gj * vj[u];
        aq = sx ? 2 * fx : -2 * fx;
        a = make_float2(__ll2float_rn(aq) * scale_q, sx ? -1.f : 1.f);   // as the GEMM epilogue
      }
      ax[k] = aq;
      as[k] = a;
    }
  }
}

cudaError_t launch_fields_inc(const DevPtrs& P, cudaStream_t s) {
  k_fields_inc<<<P.B, 256, 0, s>>>(P);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- per-search bound

__global__ void __launch_bounds__(128, 10) k_bound(DevPtrs P) {
  const int b = blockIdx.x;
  if (!P.active[b]) {
    if (threadIdx.x == 0) {
      P.surv_cnt[b] = 0;
    }
    if (P.mode != QIS_FP64 && P.dense_ctl)
      for (int g = threadIdx.x; g < P.NP / 32; g += blockDim.x)
        P.sctl[(long long)b * (P.NP / 32) + g] = make_float4(-INFINITY, 0.f, 0.f, 0.f);
    return;
  }
  const InstDesc d = P.inst[b / P.R];
  const long long base = (long long)b * P.K1;
  const int n = d.n;
  const bool fp64 = P.mode == QIS_FP64;
  extern __shared__ unsigned long long subkey[];     // [kSubMax] (u32 keys reuse the front)
  __shared__ int hist[256], hist2[256];
  __shared__ int sites[kSubSites];
  __shared__ int s_nsites, s_n2, s_bin, s_bin2, s_near, s_ns;
  __shared__ float s_thr;
  __shared__ double s_T, s_cap;
  const int cnt = P.lst_count[b];
  // key of T, the last kept energy (its value is formed by thread 0 alone: FP64 arithmetic
  // runs on a narrow pipe)
  const unsigned long long kT = (cnt == P.K1) ? P.lst_key[base + P.K1 - 1] : 0ull;
  // the parent's energy: FP64 in the FP64 mode, the exact integer E 2^q in the split modes
  // (one register for either)
  const long long epw = fp64 ? __double_as_longlong(P.par_E[b]) : P.par_q[b];
  const double Ep = __longlong_as_double(epw);   // FP64 mode
  const long long Epq = epw;                     // split modes
  const double* a64 = P.a64 + (long long)b * P.NP;
  // {a_i, s_i} of the search, staged once (split modes): every pass below reads shared memory;
  // the range of a_i is taken on the way (a ~ fl32 of the exact value in FP64 mode too: only
  // used to bin sites)
  // [NP], after the subset values: kSubMax FP64 keys in the FP64 mode, kSubMax floats otherwise
  float2* as = reinterpret_cast<float2*>(subkey + (fp64 ? kSubMax : kSubMax / 2));
  // then the parent's words and the minimum a_j of each 32-column group (sized by the context)
  uint64_t* pb = reinterpret_cast<uint64_t*>(as + P.NP);     // [Wmax]
  float* gmin = reinterpret_cast<float*>(pb + P.Wmax);        // [NP / 32]
  __shared__ float wmn[4], wmx[4];
  {
    float mn = INFINITY, mx = -INFINITY;
    if (!fp64) {
      const float2* g = P.as32 + (long long)b * P.NP;
      for (int i0 = 0; i0 < n; i0 += 8 * 128) {   // eight loads in flight per thread, then stores
        float2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int i = i0 + u * 128 + threadIdx.x;
          v[u] = (i < n) ? g[i] : make_float2(INFINITY, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int i = i0 + u * 128 + threadIdx.x;
          if (i < n) {
            as[i] = v[u];
            mn = fminf(mn, v[u].x);
            mx = fmaxf(mx, v[u].x);
          }
        }
      }
    } else {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {   // a as floats too: only used to bin sites
        const float v = (float)a64[i];
        as[i] = make_float2(v, 0.f);
        mn = fminf(mn, v);
        mx = fmaxf(mx, v);
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
      wmn[threadIdx.x >> 5] = mn;
      wmx[threadIdx.x >> 5] = mx;
    }
  }
  for (int w = threadIdx.x; w < d.W; w += blockDim.x) pb[w] = P.par_bits[(long long)b * P.Wmax + w];
  if (threadIdx.x == 0) {
    s_ns = 0;   // survivors: the singles listed below (one block per search: counted in shared memory)
    s_nsites = 0;
    s_n2 = 0;
    s_near = 0;
  }
  __syncthreads();
  if (fp64) {
    // FP64 mode: min_i a_i exactly, for the scan's row bound
    __shared__ double wmn64[4];
    double mn = INFINITY;
    for (int i = threadIdx.x; i < n; i += blockDim.x) mn = fmin(mn, a64[i]);
    for (int o = 16; o > 0; o >>= 1) mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    if ((threadIdx.x & 31) == 0) wmn64[threadIdx.x >> 5] = mn;
    __syncthreads();
    if (threadIdx.x == 0) {
      double m = wmn64[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmin(m, wmn64[w]);
      P.amin64[b] = m;
    }
  }
  const float amin = fminf(fminf(wmn[0], wmn[1]), fminf(wmn[2], wmn[3]));
  const float amax = fmaxf(fmaxf(wmx[0], wmx[1]), fmaxf(wmx[2], wmx[3]));
  // kept states one or two flips away from the parent: the only candidates that can be
  // duplicates, each equal to exactly one candidate (the kept states are the list slots
  // 0 .. cnt-1; the parent's words are in shared memory by now). Their candidate indices go
  // to dup_c for the merge's duplicate test; among the K+1+near lowest candidates at least
  // K+1 are new states.
  for (int r = threadIdx.x; r < cnt; r += blockDim.x) {
    const long long c = near_code_batched(P.lst_bits + (base + r) * P.Wmax, pb, d.W, n);
    if (c >= 0) P.dup_c[base + atomicAdd(&s_near, 1)] = (uint32_t)c;
  }
  __syncthreads();
  if (threadIdx.x == 0) P.dup_n[b] = s_near;
  const int k = P.K1 + s_near;
  double U = INFINITY;   // FP64 mode
  float Uf = INFINITY;   // split modes
  // candidates of the flip set: n singles; nu nd exchanges (nu up, nd = n - nu down spins);
  // or n singles and n(n-1)/2 pairs
  const int fl = P.flips;
  const bool ex = fl == QIS_FLIPS_EXCHANGE;
  int nu = 0;
  if (ex)
    for (int w = 0; w < d.W; ++w) nu += __popcll(pb[w]);   // bits above n are zero
  const long long C = fl == QIS_FLIPS_SINGLE ? (long long)n
                      : ex ? (long long)nu * (n - nu) : (long long)n * (n + 1) / 2;
  if (C > k && k <= kSubMax) {
    // a subset of the candidates with at least min(3k, kSubMax) members, built from low-a
    // sites found with a 256-bin histogram of a (one histogram per spin for exchanges):
    //   singles and pairs: the m lowest sites, m + m(m-1)/2 >= want, m <= kSubSites;
    //   singles only: the sites up to the bin of the k-th lowest (their a_i, <= kSubMax);
    //   exchanges: the mu lowest up and md lowest down sites, mu md >= want, every up-down
    //   pair (all of them in the flip set), mu + md <= kSubSites.
    // Any subset gives an upper bound of the k-th lowest candidate energy.
    const int want = min(3 * k, kSubMax);
    int t0 = 0, t1 = 0;
    if (fl == QIS_FLIPS_SINGLE) {
      t0 = k;
    } else if (ex) {
      const int nd = n - nu;   // nu, nd >= 1: C > k >= 1
      int m0 = max(1, (int)sqrtf((float)want));   // smallest m0 with m0^2 >= want
      while (m0 * m0 < want) ++m0;
      while (m0 > 1 && (m0 - 1) * (m0 - 1) >= want) --m0;
      int mu = min(nu, m0);
      int md = min(nd, (want + mu - 1) / mu);
      mu = min(nu, (want + md - 1) / md);
      if (mu + md > kSubSites) {
        if (mu <= kSubSites / 2) md = kSubSites - mu;
        else if (md <= kSubSites / 2) mu = kSubSites - md;
        else mu = md = kSubSites / 2;
      }
      t0 = mu;
      t1 = md;
    } else {
      // smallest m with m + m(m-1)/2 = m(m+1)/2 >= want (closed form, then a step either
      // way), at most n
      int m = max(1, (int)((sqrtf(8.f * (float)want + 1.f) - 1.f) * 0.5f));
      while (m * (m + 1) / 2 < want) ++m;
      while (m > 1 && (m - 1) * m / 2 >= want) --m;
      t0 = min(min(m, n), kSubSites);
    }
    const int lim0 = ex ? kSubSites - t1 : kSubSites;   // site slots of the first class
    const float span = fmaxf(amax - amin, 1e-30f);
    const float scale = 255.99f / span;
    auto bin_of = [&](int i) { return min(255, (int)((as[i].x - amin) * scale)); };   // both modes stage a
    for (int t = threadIdx.x; t < 256; t += blockDim.x) {
      hist[t] = 0;
      hist2[t] = 0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      atomicAdd(&((ex && sigma_of(pb, i)) ? hist2 : hist)[bin_of(i)], 1);
    __syncthreads();
    if (threadIdx.x < 32) {
      int bin, within;
      find_bin(hist, t0 - 1, bin, within);   // bin of the t0-th lowest a_i (of its class)
      if (threadIdx.x == 0) s_bin = bin;
      if (ex) {
        find_bin(hist2, t1 - 1, bin, within);
        if (threadIdx.x == 0) s_bin2 = bin;
      }
    }
    __syncthreads();
    // collect the sites (singles only: their candidate energies, in the scan's arithmetic,
    // with their range per thread)
    float vlo = INFINITY, vhi = -INFINITY;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int c = ex ? sigma_of(pb, i) : 0;
      if (bin_of(i) > (c ? s_bin2 : s_bin)) continue;
      const int slot = atomicAdd(c ? &s_n2 : &s_nsites, 1);
      if (fl == QIS_FLIPS_SINGLE) {
        if (slot < kSubMax) {
          if (fp64) {
            subkey[slot] = dkey(__dadd_rn(Ep, a64[i]));
          } else {
            const float de = as[i].x;
            vlo = fminf(vlo, de);
            vhi = fmaxf(vhi, de);
            reinterpret_cast<float*>(subkey)[slot] = de;
          }
        }
      } else if (slot < (c ? t1 : lim0)) {
        sites[c ? lim0 + slot : slot] = i;
      }
    }
    __syncthreads();
    const int mm = min(s_nsites, lim0), m2 = min(s_n2, t1);
    const int M = fl == QIS_FLIPS_SINGLE ? min(s_nsites, kSubMax) : ex ? mm * m2 : mm + mm * (mm - 1) / 2;
    // site pair of subset member t (t < M; not for single flips, whose members are written above)
    auto member = [&](int t, int& i, int& j) {
      j = -1;
      if (ex) {
        i = sites[t / m2];
        j = sites[lim0 + t % m2];
      } else if (t < mm) {
        i = sites[t];
      } else {
        // pair rank r -> (x, y), x < y < mm: row x starts at x mm - x(x+1)/2 (closed form,
        // then corrected by one step either way)
        const int r = t - mm;
        const float q = 2.f * mm - 1.f;
        int x = (int)((q - sqrtf(fmaxf(q * q - 8.f * (float)r, 0.f))) * 0.5f);
        x = max(0, min(x, mm - 2));
        while (x > 0 && x * mm - x * (x + 1) / 2 > r) --x;
        while (x < mm - 2 && (x + 1) * mm - (x + 1) * (x + 2) / 2 <= r) ++x;
        const int y = x + 1 + (r - (x * mm - x * (x + 1) / 2));
        i = sites[x];
        j = sites[y];
      }
      if (j >= 0 && i > j) { const int tmp = i; i = j; j = tmp; }
    };
    if (M >= k && !fp64 && fl != QIS_FLIPS_SINGLE) {
      // split modes: four members per thread and pass, their coupling gathers issued together
      for (int t0 = 0; t0 < M; t0 += 4 * 128) {
        int mi[4], mj[4];
        float j4v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int t = t0 + u * 128 + threadIdx.x;
          mi[u] = 0;
          mj[u] = -1;
          j4v[u] = 0.f;
          if (t < M) {
            member(t, mi[u], mj[u]);
            if (mj[u] >= 0) j4v[u] = P.J4[d.off_mat + (long long)mi[u] * d.n_pad + mj[u]];
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int t = t0 + u * 128 + threadIdx.x;
          if (t >= M) break;
          const int i = mi[u], j = mj[u];
          float de = as[i].x;
          if (j >= 0) {
            const float2 vj = as[j];
            de = as[i].x + fmaf((sigma_of(pb, i) ? -j4v[u] : j4v[u]), vj.y, vj.x);
          }
          vlo = fminf(vlo, de);
          vhi = fmaxf(vhi, de);
          reinterpret_cast<float*>(subkey)[t] = de;
        }
      }
    }
    if (M >= k) {
#pragma unroll 2
      for (int t = threadIdx.x; t < M && fp64 && fl != QIS_FLIPS_SINGLE; t += blockDim.x) {
        int i, j;
        member(t, i, j);
        double de = a64[i];
        if (j >= 0) de = dE64(a64[i], a64[j], P.J64[d.off_mat + (long long)i * d.n_pad + j],
                              sigma_of(pb, i) ^ sigma_of(pb, j));
        subkey[t] = dkey(__dadd_rn(Ep, de));
      }
      __syncthreads();
      if (fp64) U = dkey_inv(radix_select<unsigned long long>(subkey, M, k - 1, hist));
      else Uf = value_select_upper(reinterpret_cast<const float*>(subkey), M, k - 1, hist, vlo, vhi);
    }
  }
  if (threadIdx.x == 0) {
    if (fp64) {
      const double T = (cnt != P.K1) ? INFINITY : dkey_inv(kT);
      s_T = T;
      s_cap = U;
      P.thrE[b] = T;
      P.capE[b] = U;
    } else {
      // |dE~ - dE| <= delta: a and 4J are fl32 of exact values; the scan adds one FMA
      // rounding and one subtraction rounding (factor 8 margin in the constant). Everything
      // in FP32 rounded up (an upper bound at each step; GB300's FP64 pipe is narrow):
      // T - Ep from the exact integer keys, scaled by the power of two 2^-q.
      const float tE = (cnt != P.K1) ? INFINITY
                                     : __fmul_ru(__ll2float_ru((long long)(kT ^ (1ull << 63)) - Epq), (float)d.inv_scale);
      const float t0 = fminf(tE, Uf);
      const float big = __fadd_ru(__fadd_ru(__fmul_ru(3.f, fmaxf(fabsf(amin), fabsf(amax))), d.j4max),
                                  isinf(t0) ? 0.f : fabsf(t0));
      const float delta = __fmul_ru(big, 0x1p-21f);   // exact unless subnormal: rounded up
      s_thr = fminf(__fadd_ru(tE, delta), __fadd_ru(Uf, 2.f * delta));
      P.thr32[b] = s_thr;
      P.amin32[b] = amin;
    }
  }
  __syncthreads();
  if (!fp64 && P.dense_ctl) {
    // the dense scan's control word of every 32-column group g: {thr, active, RD(min_j a_j - j4max),
    // min of a_j over the groups g .. g+7 (columns < n)}. A scan chunk of at most 8 groups
    // starting at g bounds every pair term y_ij = fl(a_j +- 4J~_ij) of row i from below by
    // RD(w - max_j |4J~_ij|) (rounding is monotone), and skips rows with c_i below it.
    const int G = P.NP / 32, lane = threadIdx.x & 31;
    for (int g = threadIdx.x >> 5; g < G; g += blockDim.x >> 5) {
      const int j = 32 * g + lane;
      float v = (j < n) ? as[j].x : INFINITY;
#pragma unroll
      for (int o = 16; o; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
      if (lane == 0) gmin[g] = v;
    }
    __syncthreads();
    const float L = __fsub_rd(amin, d.j4max);
    for (int g = threadIdx.x; g < G; g += blockDim.x) {
      float w = gmin[g];
      for (int x = g + 1; x < min(g + 8, G); ++x) w = fminf(w, gmin[x]);
      P.sctl[(long long)b * G + g] = make_float4(s_thr, 1.f, L, w);
    }
  }
  // single flips: dE_i = a_i (not candidates under exchanges)
  // (one loop per mode: no FP64 instruction, even predicated off, in the split modes' loop)
  if (P.flips != QIS_FLIPS_EXCHANGE) {
    if (fp64) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double e = __dadd_rn(Ep, a64[i]);
        if ((e < s_T) && (e <= s_cap)) {
          const int slot = atomicAdd(&s_ns, 1);
          if (slot < P.cap) P.surv[(long long)b * P.cap + slot] = surv_entry(i, -1);
        }
      }
    } else {
      const float th = s_thr;
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        if (as[i].x <= th) {
          const int slot = atomicAdd(&s_ns, 1);
          if (slot < P.cap) P.surv[(long long)b * P.cap + slot] = surv_entry(i, -1);
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) P.surv_cnt[b] = s_ns;
}

cudaError_t launch_bound(const DevPtrs& P, cudaStream_t s) {
  // the split modes keep the subset as floats: a smaller footprint, ten blocks per SM
  const size_t sm = (size_t)kSubMax * (P.mode == QIS_FP64 ? 8 : 4) + (size_t)P.NP * sizeof(float2) +
                    (size_t)P.Wmax * 8 + (size_t)(P.NP / 32) * 4;
  static size_t attr = 0;
  if (attr < sm) {
    cudaError_t e = cudaFuncSetAttribute(k_bound, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr = sm;
  }
  k_bound<<<P.B, 128, sm, s>>>(P);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- FP64 pair scan
// Plain form: E' = E_p + dE exactly as defined; survivors have E' < T and E' <= cap.
// One block per 64 x 64 tile (bi <= bj) of one instance and group of kScan64Group searches.
__global__ void __launch_bounds__(256) k_scan64(DevPtrs P, const int4* work) {
  const int4 w = work[blockIdx.x];
  const InstDesc d = P.inst[w.x];
  const int n = d.n, np = d.n_pad;
  const int i0 = w.y * kTile, j0 = w.z * kTile;
  __shared__ double Jt[kTile][kTile + 1];
  __shared__ double ar_s[kTile], ac_s[kTile];
  const double* J = P.J64 + d.off_mat;
  for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
    const int r = e >> 6, c = e & 63;
    Jt[r][c] = J[(long long)(i0 + r) * np + j0 + c];
  }
  __syncthreads();
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  const int s_end = min(P.R, (w.w + 1) * kScan64Group);
  for (int s = w.w * kScan64Group; s < s_end; ++s) {
    const int b = d.first_search + s;
    __syncthreads();
    if (!P.active[b]) continue;
    const double* a = P.a64 + (long long)b * P.NP;
    if (threadIdx.x < kTile) ar_s[threadIdx.x] = a[i0 + threadIdx.x];
    else if (threadIdx.x < 2 * kTile) ac_s[threadIdx.x - kTile] = a[j0 + threadIdx.x - kTile];
    __syncthreads();
    const double T = P.thrE[b], cap = P.capE[b], Ep = P.par_E[b], amin = P.amin64[b];
    const uint64_t wi = P.par_bits[(long long)b * P.Wmax + w.y];
    const uint64_t wj = P.par_bits[(long long)b * P.Wmax + w.z];
    const unsigned rs = (unsigned)(wi >> (ty * 4)) & 15u, cs = (unsigned)(wj >> (tx * 4)) & 15u;
    for (int r = 0; r < 4; ++r) {
      const int i = i0 + ty * 4 + r;
      const double ai = ar_s[ty * 4 + r];
      // every E' of row i is at least the same expression with a_j -> min a and 4 s_i s_j J_ij
      // -> -4 max |J| (each FP64 addition is monotone in both arguments): skip the row when
      // that lower bound already fails the test
      const double lb = __dadd_rn(Ep, __dadd_rn(__dadd_rn(ai, amin), -d.j4max64));
      if (!(lb < T) || lb > cap) continue;
      for (int c = 0; c < 4; ++c) {
        const int j = j0 + tx * 4 + c;
        if (j <= i || j >= n) continue;
        const int flip = ((rs >> r) ^ (cs >> c)) & 1;
        if (!flip && P.flips == QIS_FLIPS_EXCHANGE) continue;   // exchanges need s_i != s_j
        const double e = __dadd_rn(Ep, dE64(ai, ac_s[tx * 4 + c], Jt[ty * 4 + r][tx * 4 + c], flip));
        if (e < T && e <= cap) {
          const int slot = atomicAdd(P.surv_cnt + b, 1);
          if (slot < P.cap) P.surv[(long long)b * P.cap + slot] = surv_entry(i, j);
        }
      }
    }
  }
}

cudaError_t launch_scan64(const DevPtrs& P, const int4* work, int n_work, cudaStream_t s) {
  if (n_work <= 0) return cudaSuccess;
  k_scan64<<<n_work, 256, 0, s>>>(P, work);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- exact merge (Alg. 2)
}  // namespace qis
