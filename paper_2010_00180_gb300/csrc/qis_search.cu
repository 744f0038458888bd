// qis_search.cu -- every iteration of one search in one thread block (the fused, persistent
// form of the iteration of Alg. 3 in the split precision modes).
//
// The R searches of an instance, and the instances, share nothing until the Alg. 4 merge, so
// one block can take one search through all the iterations of a qis_iterate call without ever
// waiting for another block. Per iteration t the block runs, back to back:
//   pick    the first unused kept state in key order becomes the parent (Alg. 3)
//   fields  its exact integer fields from its generating parent's, held in the aq ring, minus
//           the flipped sites' coupling columns (the Sec. III energy algebra; a parent whose
//           generator is no longer in the ring gets them from a full row sum instead);
//           a_i = -2 s_i f_i
//   bound   filter threshold (the last kept energy and an order-statistic bound), the kept
//           states one or two flips from the parent (the only possible duplicates), singles
//   scan    pair flips dE_ij = a_i + a_j + 4 s_i s_j J_ij decided by the output-sensitive scan
//   merge   exact integer keys of the survivors, duplicates dropped, the new states ranked by
//           a counting sort over buckets of their keys (no sort), first K+1 of the old list and
//           the new states by (E, stamp)
// The kept list's order, keys, stamps and used flags, the parent's spins and {a_i, s_i} stay in
// shared memory across the iterations; the kept states' bits, the aq ring and the survivor
// buffer are in global memory (written and read by this block only, within the L2 cache).
// The first iteration's parent is picked, and its fields computed (update, or the tensor-core
// GEMM for a parent without a stored generator), by the kernels launched before this one.
// The arithmetic of every phase is that of the per-kernel form (k_bound, k_scan_sparse,
// k_merge), so the kept lists are identical bit for bit.
#include "qis_block.cuh"

namespace qis {

constexpr int kSNT = 128;          // threads of a search block
constexpr int kSW = kSNT / 32;      // its warps
constexpr int kSMinBlocks = 8;      // resident blocks per SM the register budget is set for

__host__ __device__ inline int search_pcs(int cap, int merge_cand) {
  const int pc = next_pow2(cap > 256 ? cap : 256);
  return pc < merge_cand ? pc : merge_cand;
}

// Byte offsets of the dynamic shared memory of a search block.
struct SearchLayout {
  int as, pb, okey0, okey1, ostamp, oslot0, oslot1, htab, ssv, oused, scratch, total;
  int sc;   // bytes of the scratch region
};

constexpr int kSSV = 512;   // survivors held in shared memory (more go to the global buffer)
constexpr int kMBits = 7, kMB = 1 << kMBits;   // buckets of the merge's new keys

__host__ __device__ inline int align_up(int x, int a) { return (x + a - 1) / a * a; }

__host__ __device__ inline SearchLayout search_layout(int NP, int Wmax, int K1, int cap, int merge_cand) {
  SearchLayout L;
  int o = 0;
  auto take = [&](int bytes) {
    o = align_up(o, 16);
    const int r = o;
    o += bytes;
    return r;
  };
  L.as = take(NP * 8);
  L.pb = take(Wmax * 8);
  L.okey0 = take(K1 * 8);
  L.okey1 = take(K1 * 8);
  L.ostamp = take(K1 * 8);
  L.oslot0 = take(K1 * 4);
  L.oslot1 = take(K1 * 4);
  L.htab = take(next_pow2(2 * K1) * 4);
  L.ssv = take(kSSV * 8);
  L.oused = take(K1);
  // scratch: the phases' working arrays, one phase at a time
  const int bound = 4 * 256 * 4 + kSubSites * 4;
  const int scan = 3 * NP * 4 + (2 * kSparseNB + 1) * 4;
  const int merge = search_pcs(cap, merge_cand) * 16 + (512 + kMB + kSW * (kMB + 4)) * 4;
  int sc = bound > scan ? bound : scan;
  sc = sc > merge ? sc : merge;
  L.scratch = take(sc);
  L.sc = sc;
  L.total = align_up(o, 16);
  return L;
}

// Orderable unsigned key of a float (ascending floats -> ascending keys) and its inverse.
__device__ __forceinline__ unsigned fkey(float x) {
  const unsigned u = __float_as_uint(x + 0.f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Fields of a parent without a stored generator, from scratch: fq_k = hq_k + sum_j s_j Jq_jk
// (columns coalesced), aq_k = -2 s_k fq_k. Rarely taken (out of line: the hot loop stays small).
static __device__ __noinline__ void fields_full(const DevPtrs& P, const InstDesc& d, const uint64_t* pb,
                                                long long* ax, float2* as, float& mn, float& mx) {
  const long long* Jq = P.Jq + d.off_mat;
  const float scale_q = (float)d.inv_scale;
  for (int k = threadIdx.x; k < d.n; k += blockDim.x) {
    long long acc = P.hq[d.off_vec + k];
    for (int jj = 0; jj < d.n; ++jj) {
      const long long v = Jq[(long long)jj * d.n_pad + k];
      acc += sigma_of(pb, jj) ? -v : v;
    }
    const int sx = sigma_of(pb, k);
    const long long aq = sx ? 2 * acc : -2 * acc;
    const float a = __ll2float_rn(aq) * scale_q;
    ax[k] = aq;
    as[k] = make_float2(a, sx ? -1.f : 1.f);
    mn = fminf(mn, a);
    mx = fmaxf(mx, a);
  }
}

// More kept candidates than the bucket ranking takes at once (rare): keep the K+1 lowest keys
// (ties included), compacted in place; returns their number. Out of line.
static __device__ __noinline__ int keep_lowest(unsigned long long* sk, unsigned long long* se, int nv, int K1,
                                               int* rhist, int* wsum) {
  const unsigned long long x = radix_select<unsigned long long>(sk, nv, K1 - 1, rhist);
  int kept = 0;
  for (int u0 = 0; u0 < nv; u0 += blockDim.x) {
    const int e = u0 + threadIdx.x;
    unsigned long long kk = 0, ee = 0;
    bool keep = false;
    if (e < nv) {
      kk = sk[e];
      ee = se[e];
      keep = kk <= x;
    }
    int total;
    const int pos = kept + block_exclusive_sum(keep ? 1 : 0, wsum, &total);
    if (keep) {
      sk[pos] = kk;
      se[pos] = ee;
    }
    kept += total;
    __syncthreads();
  }
  return kept;
}

// (key, entry) sort of nv candidates in place, any size (rare: more than the bucket ranking
// takes after keep_lowest, i.e. many equal keys). Out of line.
static __device__ __noinline__ void sort_pairs_any(unsigned long long* sk, unsigned long long* se, int nv) {
  const int m2 = next_pow2(nv);
  for (int x = nv + threadIdx.x; x < m2; x += blockDim.x) {
    sk[x] = ~0ull;
    se[x] = ~0ull;
  }
  __syncthreads();
  bitonic_sort_smem(sk, se, m2);
}

// Exact energy E 2^q of an initial state whose energy the search initialisation left to this
// kernel, from the exact fields of its first iteration (Eq. 1): with f = J s + h,
// sum_i s_i f_i = 2 sum_{i<j} J_ij s_i s_j + sum_i h_i s_i, so E = (sum_i s_i f_i + sum_i s_i h_i) / 2,
// and s_i f_i = -aq_i / 2. Both halvings are exact (aq_i is even; the sum is twice an integer).
// red: kSNT / 32 free words of shared memory. Out of line (once per search and run).
static __device__ __noinline__ long long initial_energy(const DevPtrs& P, const InstDesc& d, const uint64_t* pb,
                                                        const long long* aq, long long* red) {
  long long acc = 0;
  for (int i = threadIdx.x; i < d.n; i += blockDim.x) {
    const long long hq = P.hq[d.off_vec + i];
    acc += (sigma_of(pb, i) ? -hq : hq) - aq[i] / 2;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  long long tot = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
  return tot / 2;
}

// FL: flip set (QIS_FLIPS_*). One block of kSNT threads per search; n_iters >= 1.
template <int FL>
__global__ void __launch_bounds__(kSNT, kSMinBlocks) k_search(DevPtrs P, int n_iters) {
  constexpr bool EX = FL == QIS_FLIPS_EXCHANGE;
  extern __shared__ __align__(16) unsigned char smem[];
  const int b = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int K1 = P.K1, Wm = P.Wmax, NP = P.NP, cap = P.cap;
  const long long base = (long long)b * K1;
  const SearchLayout L = search_layout(NP, Wm, K1, cap, P.merge_cand);
  float2* as = reinterpret_cast<float2*>(smem + L.as);
  uint64_t* pb = reinterpret_cast<uint64_t*>(smem + L.pb);
  unsigned long long* okeyA = reinterpret_cast<unsigned long long*>(smem + L.okey0);
  unsigned long long* okeyB = reinterpret_cast<unsigned long long*>(smem + L.okey1);
  uint64_t* ostamp = reinterpret_cast<uint64_t*>(smem + L.ostamp);
  int* oslotA = reinterpret_cast<int*>(smem + L.oslot0);
  int* oslotB = reinterpret_cast<int*>(smem + L.oslot1);
  uint32_t* htab = reinterpret_cast<uint32_t*>(smem + L.htab);
  unsigned long long* ssv = reinterpret_cast<unsigned long long*>(smem + L.ssv);
  const int HT = next_pow2(2 * K1);
  uint8_t* oused = reinterpret_cast<uint8_t*>(smem + L.oused);
  unsigned char* scr = smem + L.scratch;

  __shared__ int s_sel, s_near, s_ns, s_nsites, s_n2, s_bin, s_bin2, s_nl, s_nv, s_ocut;
  __shared__ float wf[2 * kSW];
  __shared__ int s_w[33];
  __shared__ unsigned long long s_kmin, s_kmax;

  const int act0 = P.active[b];
  const InstDesc d = P.inst[b / P.R];
  const int n = d.n, W = d.W;
  const int t_first = P.iter_t[b];
  const int ring_t0 = P.ring_t0[b];
  int cnt = P.lst_count[b];
  long long Epq = P.par_q[b];
  uint64_t ph = P.par_hash[b];
  for (int r = tid; r < K1; r += kSNT) {
    okeyA[r] = P.lst_key[base + r];
    oslotA[r] = P.lst_ord[base + r];
    ostamp[r] = P.lst_stamp[base + r];
    oused[r] = P.lst_used[base + r];
  }
  for (int w = tid; w < W; w += kSNT) pb[w] = P.par_bits[(long long)b * Wm + w];
  float mn = INFINITY, mx = -INFINITY;   // this thread's range of a_i (for the bound)
  if (act0)
    for (int i = tid; i < n; i += kSNT) {
      const float2 v = P.as32[(long long)b * NP + i];
      as[i] = v;
      mn = fminf(mn, v.x);
      mx = fmaxf(mx, v.x);
    }
  __syncthreads();
  if (act0 && P.e0_pend[b]) {   // block-uniform: the list is [psi0] and psi0 is the parent
    Epq = initial_energy(P, d, pb, aq_of(P, b, t_first), reinterpret_cast<long long*>(scr));
    if (tid == 0) {
      const int s0 = oslotA[0];
      const double E0 = ldexp((double)Epq, -d.q);
      okeyA[0] = qkey(Epq);
      P.lst_q[base + s0] = Epq;
      P.lst_E[base + s0] = E0;
      P.init_q[b] = Epq;
      P.init_E[b] = E0;
      P.e0_pend[b] = 0;
    }
    __syncthreads();
  }

  int act = act0, t = t_first, cur = 0;
  int nprod = 0;
  unsigned long long npair = 0, nev = 0, nsurv = 0;
  const float scale_q = (float)d.inv_scale;
  const long long* Jq = P.Jq + d.off_mat;
  const float* J4 = P.J4 + d.off_mat;
  unsigned long long* surv = P.surv + (long long)b * cap;
  // survivor slot s: shared memory below kSSV, the search's global buffer above (up to cap)
  auto put_surv = [&](int slot, unsigned long long e) {
    if (slot < kSSV) ssv[slot] = e;
    else if (slot < cap) surv[slot] = e;
  };

  for (int iter = 0; iter < n_iters; ++iter) {
    unsigned long long* okey = cur ? okeyB : okeyA;
    unsigned long long* okeyN = cur ? okeyA : okeyB;
    int* oslot = cur ? oslotB : oslotA;
    int* oslotN = cur ? oslotA : oslotB;
    if (iter > 0) {
      t += 1;
      if (!act) continue;
      // ------------------------------------------------------------ pick (Alg. 3)
      if (warp == 0) {
        int sel = -1;
        for (int r0 = 0; r0 < cnt && sel < 0; r0 += 32) {
          const int r = r0 + lane;
          const bool un = r < cnt && !oused[oslot[r]];
          const unsigned m = __ballot_sync(0xffffffffu, un);
          if (m) sel = r0 + __ffs(m) - 1;
        }
        if (lane == 0) s_sel = sel;
      }
      __syncthreads();
      const int sel = s_sel;
      if (sel < 0) {   // every kept state used: the search ends (block-uniform)
        act = 0;
        continue;
      }
      const int pslot = oslot[sel];
      Epq = (long long)(okey[sel] ^ (1ull << 63));
      const uint64_t pst = ostamp[pslot];
      ph = P.lst_hash[base + pslot];
      for (int w = tid; w < W; w += kSNT) pb[w] = P.lst_bits[(base + pslot) * Wm + w];
      __syncthreads();   // the parent's words; every thread has read s_sel and the used flags
      if (tid == 0) {
        oused[pslot] = 1;
        P.lst_used[base + pslot] = 1;
      }
      ++nprod;
      if (FL == QIS_FLIPS_SINGLE_PAIR) npair += (unsigned long long)n * (n - 1) / 2;
      if (EX) {
        int down = 0;
        for (int w = 0; w < W; ++w) down += __popcll(pb[w]);
        npair += (unsigned long long)down * (unsigned long long)(n - down);
      }
      // ------------------------------------------------------------ fields
      // x = the parent, entered at iteration tg as candidate c of that iteration's parent g
      const int tg = (int)(pst >> 32);
      long long* __restrict__ ax = aq_of(P, b, t);
      if (tg >= 1 && tg > ring_t0 && tg < t && t - tg < P.ring_n) {
        int i, j;
        decode_candidate(n, (uint32_t)pst, i, j);
        const long long* __restrict__ ag = aq_of(P, b, tg);
        const long long* __restrict__ Ji = Jq + (long long)i * d.n_pad;   // row i = column i
        const long long* __restrict__ Jj = Jq + (long long)max(j, 0) * d.n_pad;
        // one site per thread and pass, pipelined: the next site's three loads are issued before
        // the current site's fields are formed. With s_g = -s_x at the flipped sites i, j,
        //   aq_x,k = s_x,k s_g,k aq_g,k + 4 s_x,k (s_g,i Jq_ik + s_g,j Jq_jk),
        // s_g,i = +1 where the parent's bit i is set (exact int64)
        const bool pi = sigma_of(pb, i) != 0;
        const bool pj = j >= 0 && sigma_of(pb, j) != 0;
        long long g_n = 0, i_n = 0, j_n = 0;
        auto load = [&](int k) {
          if (k < n) {
            g_n = ag[k];
            i_n = Ji[k];
            if (j >= 0) j_n = Jj[k];
          }
        };
        load(tid);
#pragma unroll 1
        for (int k = tid; k < n; k += kSNT) {
          const long long vg = g_n, vi = i_n, vj = j_n;
          load(k + kSNT);
          const int sx = sigma_of(pb, k);
          const long long tt = (pi ? vi : -vi) + (j >= 0 ? (pj ? vj : -vj) : 0);
          const long long aq = ((k == i || k == j) ? -vg : vg) + (sx ? -4 * tt : 4 * tt);
          const float a = __ll2float_rn(aq) * scale_q;
          ax[k] = aq;
          as[k] = make_float2(a, sx ? -1.f : 1.f);
          mn = fminf(mn, a);
          mx = fmaxf(mx, a);
        }
      } else {
        fields_full(P, d, pb, ax, as, mn, mx);   // no stored generator
      }
    } else if (!act) {
      continue;
    }
    // ---------------------------------------------------------------- bound
    // range of a over the block; the kept states one or two flips from the parent (their
    // candidate indices: the only candidates that can be duplicates, each equal to exactly one)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if (lane == 0) {
      wf[warp] = mn;
      wf[kSW + warp] = mx;
    }
    if (tid == 0) {
      s_near = 0;
      s_ns = 0;
      s_nsites = 0;
      s_n2 = 0;
      s_nl = 0;
      s_nv = 0;
      s_ocut = cnt;
      s_kmin = ~0ull;
      s_kmax = 0;
    }
    for (int x = tid; x < HT; x += kSNT) htab[x] = kNoCand;
    {
      int* hist = reinterpret_cast<int*>(scr);   // the bound's histograms, cleared for this iteration
      for (int x = tid; x < 4 * 256; x += kSNT) hist[x] = 0;
    }
    __syncthreads();   // the fields and the range are complete
    float amin = wf[0], amax = wf[kSW];
#pragma unroll
    for (int w = 1; w < kSW; ++w) {
      amin = fminf(amin, wf[w]);
      amax = fmaxf(amax, wf[kSW + w]);
    }
    mn = INFINITY;
    mx = -INFINITY;
    for (int r = tid; r < cnt; r += kSNT) {
      const long long c = near_code_sp(P.lst_bits + (base + r) * Wm, pb, W, n);
      if (c >= 0) {
        atomicAdd(&s_near, 1);
        uint32_t pos = chash((uint32_t)c) & (HT - 1);
        while (atomicCAS(&htab[pos], kNoCand, (uint32_t)c) != kNoCand) pos = (pos + 1) & (HT - 1);
      }
    }
    __syncthreads();
    const int ndup = s_near;
    const int k = K1 + ndup;
    float Uf = INFINITY;
    int nu = 0;
    if (EX)
      for (int w = 0; w < W; ++w) nu += __popcll(pb[w]);
    const long long Ccand = FL == QIS_FLIPS_SINGLE ? (long long)n : EX ? (long long)nu * (n - nu) : (long long)n * (n + 1) / 2;
    if (Ccand > k && k <= kSubMax) {
      // the bound's histograms (cleared before the fields barrier): site bins, the second spin
      // class's site bins (exchanges), the subset values' counts and their per-bin maxima
      int* hist = reinterpret_cast<int*>(scr);                        // [256]
      int* hist2 = hist + 256;                                         // [256]
      int* vhist = hist2 + 256;                                        // [256]
      unsigned* vmax = reinterpret_cast<unsigned*>(vhist + 256);       // [256]
      int* sites = reinterpret_cast<int*>(vmax + 256);                 // [kSubSites]
      const int want = min(3 * k, kSubMax);
      int t0 = 0, t1 = 0;
      if (FL == QIS_FLIPS_SINGLE) {
        t0 = k;
      } else if (EX) {
        const int nd = n - nu;
        int m0 = max(1, (int)sqrtf((float)want));
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
        int m = max(1, (int)((sqrtf(8.f * (float)want + 1.f) - 1.f) * 0.5f));
        while (m * (m + 1) / 2 < want) ++m;
        while (m > 1 && (m - 1) * m / 2 >= want) --m;
        t0 = min(min(m, n), kSubSites);
      }
      const int lim0 = EX ? kSubSites - t1 : kSubSites;
      const float scale = 255.99f / fmaxf(amax - amin, 1e-30f);
      auto bin_of = [&](int i) { return min(255, (int)((as[i].x - amin) * scale)); };
      for (int i = tid; i < n; i += kSNT) atomicAdd(&((EX && sigma_of(pb, i)) ? hist2 : hist)[bin_of(i)], 1);
      __syncthreads();
      if (warp == 0) {
        int bin, within;
        find_bin(hist, t0 - 1, bin, within);
        if (lane == 0) s_bin = bin;
        if (EX) {
          find_bin(hist2, t1 - 1, bin, within);
          if (lane == 0) s_bin2 = bin;
        }
      }
      __syncthreads();
      // the subset's values are binned as they are formed, over a range that holds them: every
      // selected site has a below the upper edge of its class's cut bin (one bin of margin for
      // the rounding of the binning), a pair lies within 4 max|J~| of a_i + a_j (values outside
      // clamp to the end bins, which keeps the binning monotone)
      const float cut0 = __fadd_ru(amin, __fdiv_ru((float)(s_bin + 2), scale));
      const float cut1 = EX ? __fadd_ru(amin, __fdiv_ru((float)(s_bin2 + 2), scale)) : cut0;
      const float hi_v = FL == QIS_FLIPS_SINGLE ? cut0 : __fadd_ru(__fadd_ru(cut0, cut1), d.j4max);
      const float lo_b = FL == QIS_FLIPS_SINGLE ? amin : __fsub_rd(__fadd_rd(amin, amin), d.j4max);
      const float scale_v = 255.99f / fmaxf(hi_v - lo_b, 1e-30f);
      auto put_value = [&](float v) {
        const int bin = min(255, max(0, (int)((v - lo_b) * scale_v)));
        atomicAdd(&vhist[bin], 1);
        atomicMax(&vmax[bin], fkey(v));
      };
      for (int i = tid; i < n; i += kSNT) {
        const int c = EX ? sigma_of(pb, i) : 0;
        if (bin_of(i) > (c ? s_bin2 : s_bin)) continue;
        const int slot = atomicAdd(c ? &s_n2 : &s_nsites, 1);
        if (FL == QIS_FLIPS_SINGLE) {
          if (slot < kSubMax) put_value(as[i].x);
        } else if (slot < (c ? t1 : lim0)) {
          sites[c ? lim0 + slot : slot] = i;
        }
      }
      __syncthreads();
      const int mm = min(s_nsites, lim0), m2 = min(s_n2, t1);
      const int M = FL == QIS_FLIPS_SINGLE ? min(s_nsites, kSubMax) : EX ? mm * m2 : mm + mm * (mm - 1) / 2;
      auto member = [&](int q, int& i, int& j) {   // exchanges: (class 0 site, class 1 site)
        i = sites[q / m2];
        j = sites[lim0 + q % m2];
        if (i > j) {
          const int tmp = i;
          i = j;
          j = tmp;
        }
      };
      if (M >= k && FL != QIS_FLIPS_SINGLE) {
        if (!EX) {
          // the subset's singles, then its pairs row by row: warp w takes the rows x = w, w + 4,
          // ..., its lanes the partners y > x (no index decoding; a warp reads one row of 4J~)
          for (int q = tid; q < mm; q += kSNT) put_value(as[sites[q]].x);
          for (int x = warp; x < mm; x += kSW) {
            const int sx = sites[x];
            for (int y = x + 1 + lane; y < mm; y += 32) {
              const int sy = sites[y];
              const int i = min(sx, sy), j = max(sx, sy);
              const float j4 = J4[(long long)i * d.n_pad + j];
              const float2 vj = as[j];
              put_value(as[i].x + fmaf((sigma_of(pb, i) ? -j4 : j4), vj.y, vj.x));
            }
          }
        } else {
          for (int q0 = 0; q0 < M; q0 += kSNT) {   // exchanges: pair q of the cross product
            const int q = q0 + tid;
            int i = 0, j = -1;
            float j4 = 0.f;
            if (q < M) {
              member(q, i, j);
              j4 = J4[(long long)i * d.n_pad + j];
            }
            if (q >= M) continue;
            const float2 vj = as[j];
            put_value(as[i].x + fmaf((sigma_of(pb, i) ? -j4 : j4), vj.y, vj.x));
          }
        }
      }
      if (M >= k) {
        // U = the largest subset value in the bins up to the one holding the k-th smallest
        // (binning is monotone, so at least k subset values are <= U): every warp alike
        __syncthreads();
        int bsel, within;
        find_bin(vhist, k - 1, bsel, within);
        unsigned mk = 0u;
        for (int x = lane; x <= bsel; x += 32) mk = max(mk, vmax[x]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mk = max(mk, __shfl_xor_sync(0xffffffffu, mk, o));
        Uf = fkey_inv(mk);
      }
    }
    float thr;
    {
      // |dE~ - dE| <= delta: a and 4J are fl32 of exact values; the scan adds one FMA rounding
      // and one subtraction rounding (factor 8 margin). Everything in FP32 rounded up; T - Ep
      // from the exact integer keys, scaled by the power of two 2^-q. (Every thread forms the
      // same value from the same operands.)
      const unsigned long long kT = okey[K1 - 1];
      const float tE = (cnt != K1) ? INFINITY
                                   : __fmul_ru(__ll2float_ru((long long)(kT ^ (1ull << 63)) - Epq), scale_q);
      const float tt = fminf(tE, Uf);
      const float big = __fadd_ru(__fadd_ru(__fmul_ru(3.f, fmaxf(fabsf(amin), fabsf(amax))), d.j4max),
                                  isinf(tt) ? 0.f : fabsf(tt));
      const float delta = __fmul_ru(big, 0x1p-21f);
      thr = fminf(__fadd_ru(tE, delta), __fadd_ru(Uf, 2.f * delta));
    }
    // single flips: dE_i = a_i (not candidates under exchanges; with pairs, tested in the
    // live-row pass below)
    if (FL == QIS_FLIPS_SINGLE) {
      for (int i = tid; i < n; i += kSNT) {
        if (as[i].x <= thr) {
          const int slot = atomicAdd(&s_ns, 1);
          put_surv(slot, surv_entry(i, -1));
        }
      }
    }
    // ---------------------------------------------------------------- scan (pairs)
    if (FL != QIS_FLIPS_SINGLE) {
      int* li = reinterpret_cast<int*>(scr);   // [NP] live rows
      int* pc = li + NP;                       // [NP] their rm, then list offsets
      int* cj = pc + NP;                       // [NP] columns in bucket order
      int* bs = cj + NP;                       // [kSparseNB + 1]
      int* bcur = bs + kSparseNB + 1;          // [kSparseNB]
      // the row of each pair, while the pairs fit the rest of the scratch
      unsigned short* rowof = reinterpret_cast<unsigned short*>(bcur + kSparseNB);
      const int rcap = (L.sc - (3 * NP + 2 * kSparseNB + 1) * 4) / 2;
      const float* rm = P.rm4 + d.off_vec;
      __syncthreads();   // the bound's scratch is free
      for (int x = tid; x < kSparseNB; x += kSNT) bcur[x] = 0;
      float bl = -INFINITY;
      constexpr int SB = 5;
      for (int i0 = 0; i0 < n; i0 += SB * kSNT) {
        float r[SB];
#pragma unroll
        for (int u = 0; u < SB; ++u) {
          const int i = i0 + tid + u * kSNT;
          r[u] = (i < n) ? rm[i] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < SB; ++u) {
          const int i = i0 + tid + u * kSNT;
          if (i < n) {
            const float ai = as[i].x;
            if (!EX && ai <= thr) put_surv(atomicAdd(&s_ns, 1), surv_entry(i, -1));
            const float c = __fsub_rn(thr, ai);
            if (c >= __fsub_rd(amin, r[u])) {
              const int q = atomicAdd(&s_nl, 1);
              li[q] = i;
              pc[q] = __float_as_int(r[u]);
              bl = fmaxf(bl, __fadd_ru(nextafterf(c, INFINITY), r[u]));
            }
          }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) bl = fmaxf(bl, __shfl_xor_sync(0xffffffffu, bl, o));
      if (lane == 0) wf[warp] = bl;
      __syncthreads();
      const int nl = s_nl;
      if (nl > 0) {   // block-uniform
        float B = wf[0];
#pragma unroll
        for (int w = 1; w < kSW; ++w) B = fmaxf(B, wf[w]);
        const float span = __fsub_ru(B, amin);
        const float inv = (span > 0.f && span < INFINITY) ? __fdiv_rn((float)kSparseNB, span) : 0.f;
        for (int j = tid; j < n; j += kSNT)
          if (as[j].x < B) atomicAdd(&bcur[sparse_bucket(as[j].x, amin, inv)], 1);
        __syncthreads();
        if (warp == 0) {
          int x[kSparseNB / 32], s = 0;
#pragma unroll
          for (int q = 0; q < kSparseNB / 32; ++q) {
            x[q] = bcur[lane * (kSparseNB / 32) + q];
            s += x[q];
          }
          int inc = s;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
          }
          int acc = inc - s;
#pragma unroll
          for (int q = 0; q < kSparseNB / 32; ++q) {
            bs[lane * (kSparseNB / 32) + q] = acc;
            bcur[lane * (kSparseNB / 32) + q] = acc;
            acc += x[q];
          }
          if (lane == 31) bs[kSparseNB] = acc;
        }
        __syncthreads();
        // site code in place of s_j: (position in the column order << 1) | sigma_j, or INT_MIN |
        // sigma_j for a site at or above B
        for (int j = tid; j < n; j += kSNT) {
          const float2 v = as[j];
          const int sg = v.y < 0.f;
          int code = INT_MIN | sg;
          if (v.x < B) {
            const int q = atomicAdd(&bcur[sparse_bucket(v.x, amin, inv)], 1);
            cj[q] = j;
            code = (q << 1) | sg;
          }
          as[j].y = __int_as_float(code);
        }
        for (int q = tid; q < nl; q += kSNT) {
          const int i = li[q];
          const float c = __fsub_rn(thr, as[i].x), rr = __int_as_float(pc[q]);
          pc[q] = bs[sparse_bucket(__fadd_ru(nextafterf(c, INFINITY), rr), amin, inv) + 1];
        }
        __syncthreads();
        {
          const int per = (nl + kSNT - 1) / kSNT, q0 = min(nl, tid * per), q1 = min(nl, q0 + per);
          int sum = 0;
          for (int q = q0; q < q1; ++q) {
            const int code = __float_as_int(as[li[q]].y);
            const int x = code < 0 ? 0 : max(0, pc[q] - (code >> 1) - 1);
            pc[q] = x;
            sum += x;
          }
          int inc = sum;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
          }
          if (lane == 31) s_w[warp] = inc;
          __syncthreads();
          int acc = inc - sum;
          for (int w = 0; w < warp; ++w) acc += s_w[w];
          for (int q = q0; q < q1; ++q) {
            const int x = pc[q];
            pc[q] = acc;
            for (int e = acc, e1 = min(acc + x, rcap); e < e1; ++e) rowof[e] = (unsigned short)q;
            acc += x;
          }
        }
        __syncthreads();
        int tot = 0;
#pragma unroll
        for (int w = 0; w < kSW; ++w) tot += s_w[w];
        const bool direct = tot <= rcap;   // every pair's row in rowof (block-uniform)
        // one pair per thread and pass, pipelined: the coupling load of the next pass's pair is
        // issued before the current pair is tested
        int ij_n = 0;
        float cv_n = 0.f, av_n = 0.f, jv_n = 0.f;
        bool ok_n = false, neg_n = false;
        auto stage = [&](int e) {
          ok_n = false;
          if (e < tot) {
            int lo = 0;
            if (direct) {
              lo = rowof[e];
            } else {
              int hi = nl;
              while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (pc[mid] <= e) lo = mid; else hi = mid;
              }
            }
            const int i = li[lo];
            const float2 vi = as[i];
            const int ci = __float_as_int(vi.y);
            const int j = cj[(ci >> 1) + 1 + e - pc[lo]];
            const float2 vj = as[j];
            ij_n = min(i, j) | (max(i, j) << 16);
            neg_n = ((ci ^ __float_as_int(vj.y)) & 1) != 0;
            cv_n = __fsub_rn(thr, vi.x);
            av_n = vj.x;
            ok_n = !EX || neg_n;
            if (ok_n) jv_n = J4[(long long)i * d.n_pad + j];
          }
        };
        stage(tid);
        for (int u0 = 0; u0 < tot; u0 += kSNT) {
          const int ij = ij_n;
          const float cv = cv_n, av = av_n, jv = jv_n;
          const bool ok = ok_n, neg = neg_n;
          stage(u0 + kSNT + tid);
          bool hit = false;
          if (ok) {
            ++nev;
            hit = fmaf(neg ? -1.f : 1.f, jv, av) <= cv;
          }
          const unsigned m = __ballot_sync(0xffffffffu, hit);
          if (m) {
            const int leader = __ffs(m) - 1;
            int sb = 0;
            if (lane == leader) sb = atomicAdd(&s_ns, __popc(m));
            sb = __shfl_sync(0xffffffffu, sb, leader);
            const int slot = sb + __popc(m & ((1u << lane) - 1u));
            if (hit) put_surv(slot, surv_entry(ij & 0xffff, ij >> 16));
          }
        }
      }
    }
    // ---------------------------------------------------------------- merge (Alg. 2)
    unsigned long long* sk = reinterpret_cast<unsigned long long*>(scr);
    const int PCs = search_pcs(cap, P.merge_cand);
    unsigned long long* se = sk + PCs;
    // after the keys: mem [256] candidates by bucket, rank [256], bucket sizes [kMB], every
    // warp's bucket starts [kSW][kMB + 4]; keep_lowest's histogram overlaps the starts only
    int* mem = reinterpret_cast<int*>(se + PCs);
    int* bcnt = mem + 512;
    int* rhist = bcnt + 2 * kMB;                     // [256] (keep_lowest, before the buckets)
    __syncthreads();   // every survivor written; the scan's scratch is free
    for (int x = tid; x < kMB; x += kSNT) bcnt[x] = 0;
    const int S = s_ns;
    if (S > cap) {   // block-uniform: the buffer held only the first cap survivors
      if (tid == 0) atomicOr(P.status, kStatCapacity);
      act = 0;
      continue;
    }
    nsurv += (unsigned long long)S;
    const bool big = S > PCs;
    if (big) {
      const long long stride = next_pow2(max(cap, 256));
      sk = P.mrg_scratch + (long long)b * 2 * stride;
      se = sk + stride;
    }
    const long long Tq = (cnt == K1) ? (long long)(okey[K1 - 1] ^ (1ull << 63)) : LLONG_MAX;
    const long long* aqb = aq_of(P, b, t);
    unsigned long long kmn = ~0ull, kmx = 0;
    for (int u0 = 0; u0 < S; u0 += kSNT) {
      const int e = u0 + tid;
      bool keep = false;
      unsigned long long kk = 0, ent = 0;
      if (e < S) {
        ent = (e < kSSV) ? ssv[e] : surv[e];
        int i, j;
        surv_sites(ent, i, j);
        ent |= (j < 0) ? (uint32_t)i : pair_index(n, i, j);
        long long de = aqb[i];
        if (j >= 0) {
          const long long jq = Jq[(long long)i * d.n_pad + j];
          de += aqb[j] + ((sigma_of(pb, i) ^ sigma_of(pb, j)) ? -4 * jq : 4 * jq);
        }
        const long long eq = Epq + de;
        kk = qkey(eq);
        keep = eq < Tq;   // Alg. 2: strict <
        if (keep) {
          const uint32_t c = (uint32_t)ent;
          for (uint32_t pos = chash(c) & (HT - 1); htab[pos] != kNoCand; pos = (pos + 1) & (HT - 1))
            if (htab[pos] == c) {
              keep = false;   // a kept state (the binary search of Alg. 2)
              break;
            }
        }
      }
      const unsigned bal = __ballot_sync(0xffffffffu, keep);
      if (bal) {
        int wb = 0;
        if (lane == 0) wb = atomicAdd(&s_nv, __popc(bal));
        wb = __shfl_sync(0xffffffffu, wb, 0);
        if (keep) {
          const int slot = wb + __popc(bal & ((1u << lane) - 1));
          sk[slot] = kk;
          se[slot] = ent;
          kmn = min(kmn, kk);
          kmx = max(kmx, kk);
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      kmn = min(kmn, __shfl_xor_sync(0xffffffffu, kmn, o));
      kmx = max(kmx, __shfl_xor_sync(0xffffffffu, kmx, o));
    }
    if (lane == 0 && kmn <= kmx) {
      atomicMin(&s_kmin, kmn);
      atomicMax(&s_kmax, kmx);
    }
    __syncthreads();
    int nv = s_nv;
    // more kept candidates than the buckets take at once: only the K+1 lowest can enter the list
    if (nv > 256 && nv > K1) nv = keep_lowest(sk, se, nv, K1, rhist, s_w);
    const unsigned long long kmin = s_kmin, kmax = s_kmax;
    // the new candidates' order (E, c) as one 64-bit value, (E - Emin) << cb | c, where the keys'
    // span leaves room for c (always but for extreme ranges); equal energies are ordered by c
    const uint32_t n_cand = (uint32_t)n + (uint32_t)((long long)n * (n - 1) / 2);
    const int cb = 32 - __clz((int)n_cand);
    const bool bucketed = nv <= 256 && ((kmax - kmin) >> (64 - cb)) == 0;   // block-uniform
    int* rnk = mem + 256;              // [256] place of each new candidate among the new ones
    int* bst = bcnt + kMB + warp * (kMB + 4);   // this warp's bucket starts [kMB + 1]
    const int sh = max(0, 64 - __clzll((long long)(((kmax - kmin) << cb) | ((1ull << cb) - 1))) - kMBits);
    if (bucketed) {
      // without sorting them: the order values packed in place, a counting sort by their top
      // bits into kMB buckets, then a count within the bucket (the values are distinct)
      int wb0 = 0, wb1 = 0;
      if (tid < nv) {
        sk[tid] = ((sk[tid] - kmin) << cb) | (uint32_t)se[tid];
        wb0 = atomicAdd(&bcnt[(int)(sk[tid] >> sh)], 1);
      }
      if (tid + kSNT < nv) {
        sk[tid + kSNT] = ((sk[tid + kSNT] - kmin) << cb) | (uint32_t)se[tid + kSNT];
        wb1 = atomicAdd(&bcnt[(int)(sk[tid + kSNT] >> sh)], 1);
      }
      __syncthreads();
      {   // every warp forms the bucket starts itself (no barrier)
        int x[kMB / 32], sum = 0;
#pragma unroll
        for (int q = 0; q < kMB / 32; ++q) {
          x[q] = bcnt[lane * (kMB / 32) + q];
          sum += x[q];
        }
        int inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, inc, o);
          if (lane >= o) inc += y;
        }
        int acc = inc - sum;
#pragma unroll
        for (int q = 0; q < kMB / 32; ++q) {
          bst[lane * (kMB / 32) + q] = acc;
          acc += x[q];
        }
        if (lane == 31) bst[kMB] = acc;
        __syncwarp();
      }
      if (tid < nv) mem[bst[(int)(sk[tid] >> sh)] + wb0] = tid;
      if (tid + kSNT < nv) mem[bst[(int)(sk[tid + kSNT] >> sh)] + wb1] = tid + kSNT;
      __syncthreads();
      for (int p = tid; p < nv; p += kSNT) {
        const unsigned long long vp = sk[p];
        const int bk = (int)(vp >> sh);
        int r = bst[bk];
        for (int q = bst[bk], q1 = bst[bk + 1]; q < q1; ++q) r += (sk[mem[q]] < vp) ? 1 : 0;
        rnk[p] = r;
      }
    } else {
      sort_pairs_any(sk, se, nv);   // rare: sorted in place, the place of p is p
      for (int p = tid; p < nv; p += kSNT) rnk[p] = p;
    }
    // old entries: their place plus the new candidates strictly below their key
    for (int o = tid; o < cnt; o += kSNT) {
      const unsigned long long ko = okey[o];
      int lo;
      if (nv == 0 || ko <= kmin) {
        lo = 0;
      } else if (ko > kmax) {
        lo = nv;
      } else if (bucketed) {
        const unsigned long long vo = (ko - kmin) << cb;   // below every new value of energy ko
        const int bk = (int)(vo >> sh);
        lo = bst[bk];
        for (int q = bst[bk], q1 = bst[bk + 1]; q < q1; ++q) lo += (sk[mem[q]] < vo) ? 1 : 0;
      } else {
        lo = 0;
        int hi = nv;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (sk[mid] < ko) lo = mid + 1; else hi = mid;
        }
      }
      const int rank = o + lo;
      if (rank < K1) {
        oslotN[rank] = oslot[o];
        okeyN[rank] = ko;
      } else {
        atomicMin(&s_ocut, o);
      }
    }
    __syncthreads();
    const int ocut = s_ocut, n_ev = cnt - ocut;
    for (int p = tid; p < nv; p += kSNT) {
      const unsigned long long kp = bucketed ? (sk[p] >> cb) + kmin : sk[p];
      int lo = 0, hi = cnt;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (okey[mid] <= kp) lo = mid + 1; else hi = mid;
      }
      const int rn = rnk[p], rank = rn + lo;
      if (rank >= K1) continue;
      const int slot = (rn < n_ev) ? oslot[ocut + rn] : cnt + (rn - n_ev);
      uint32_t c;
      int i, j;
      surv_decode(se[p], c, i, j);
      uint64_t* dst = P.lst_bits + (base + slot) * Wm;
      {   // the parent's words, two per store when the rows are 16-byte aligned (fewer store
          // instructions of scattered rows than one word each), then the words of the flipped
          // sites stored again with their bits flipped (same thread and address: the later wins)
        int x = 0;
        if ((Wm & 1) == 0)
          for (; x + 1 < W; x += 2)
            *reinterpret_cast<ulonglong2*>(dst + x) = *reinterpret_cast<const ulonglong2*>(pb + x);
        for (; x < W; ++x) dst[x] = pb[x];
        const int wi = i >> 6;
        uint64_t vi = pb[wi] ^ (1ull << (i & 63));
        if (j >= 0 && (j >> 6) == wi) vi ^= 1ull << (j & 63);
        dst[wi] = vi;
        if (j >= 0 && (j >> 6) != wi) dst[j >> 6] = pb[j >> 6] ^ (1ull << (j & 63));
      }
      const uint64_t stamp = ((uint64_t)t << 32) | c;
      P.lst_q[base + slot] = (long long)(kp ^ (1ull << 63));
      P.lst_stamp[base + slot] = stamp;
      ostamp[slot] = stamp;
      P.lst_hash[base + slot] = ph ^ P.zob[i] ^ ((j >= 0) ? P.zob[j] : 0ull);
      P.lst_used[base + slot] = 0;
      oused[slot] = 0;
      oslotN[rank] = slot;
      okeyN[rank] = kp;
    }
    cnt = min(K1, cnt + nv);
    cur ^= 1;
    __syncthreads();   // the new order is complete before the next pick reads it
  }
  // ------------------------------------------------------------------ write back
  const unsigned long long* okey = cur ? okeyB : okeyA;
  const int* oslot = cur ? oslotB : oslotA;
  for (int r = tid; r < cnt; r += kSNT) {
    P.lst_key[base + r] = okey[r];
    P.lst_ord[base + r] = oslot[r];
  }
  if (act0) {   // the last parent (what the per-kernel form leaves in these fields)
    for (int w = tid; w < W; w += kSNT) P.par_bits[(long long)b * Wm + w] = pb[w];
  }
  if (tid == 0) {
    P.lst_count[b] = cnt;
    P.iter_t[b] = t_first + n_iters - 1;
    if (act0) {
      P.active[b] = act;
      P.par_q[b] = Epq;
      P.par_hash[b] = ph;
      P.nprod[b] += nprod;
      P.npair[b] += npair;
      if (nsurv) atomicAdd(P.surv_tot + (b & 63), nsurv);
    }
  }
  if (act0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nev += __shfl_xor_sync(0xffffffffu, nev, o);
    if (lane == 0 && nev) atomicAdd(P.eval_cnt + (b & 63), nev);
  }
}

size_t search_smem(const DevPtrs& P) { return (size_t)search_layout(P.NP, P.Wmax, P.K1, P.cap, P.merge_cand).total; }

cudaError_t launch_search(const DevPtrs& P, int n_iters, cudaStream_t s) {
  if (n_iters <= 0 || P.B == 0) return cudaSuccess;
  const size_t sm = search_smem(P);
  static size_t attr[3] = {0, 0, 0};
  const int fl = P.flips;
  if (attr[fl] < sm) {
    cudaError_t e = fl == QIS_FLIPS_SINGLE ? cudaFuncSetAttribute(k_search<QIS_FLIPS_SINGLE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)
                  : fl == QIS_FLIPS_EXCHANGE ? cudaFuncSetAttribute(k_search<QIS_FLIPS_EXCHANGE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)
                                             : cudaFuncSetAttribute(k_search<QIS_FLIPS_SINGLE_PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr[fl] = sm;
  }
  if (fl == QIS_FLIPS_SINGLE) k_search<QIS_FLIPS_SINGLE><<<P.B, kSNT, sm, s>>>(P, n_iters);
  else if (fl == QIS_FLIPS_EXCHANGE) k_search<QIS_FLIPS_EXCHANGE><<<P.B, kSNT, sm, s>>>(P, n_iters);
  else k_search<QIS_FLIPS_SINGLE_PAIR><<<P.B, kSNT, sm, s>>>(P, n_iters);
  return cudaGetLastError();
}

}  // namespace qis
