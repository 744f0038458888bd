// qis_merge.cu -- the exact list update of one iteration (Alg. 2), one block per search.
//
// Input: the survivor buffer of the search (entries {i, j} of the single flips from k_bound
// and of the pairs that passed the scan's filter; the candidate index c is added here).
// Output: the new kept list.
//
//  1. Every candidate gets its exact energy: in the split modes from exact fixed-point
//     integers, E'q = E_pq + aq_i (+ aq_j + 4 s_i s_j Jq_ij), compared as integers with the
//     integer energies of the kept states (no floating point on this path); in the FP64 mode
//     with the defining FP64 arithmetic. Candidates with E' >= T (the last kept energy, Alg. 2: strict
//     <) are dropped, as are duplicates of a kept state (the binary search of Alg. 2): a kept
//     state equals a candidate only if it is one or two flips from the parent, and then it
//     is exactly the candidate of those flips, so duplicates are found by candidate index.
//  2. The kept candidates are sorted by (E, c): warp-sorted runs of 32 merged by rank (binary
//     search in the other runs) for up to 256 candidates, a shared-memory bitonic network beyond.
//  3. New list = first K+1 of (old list, new candidates) by (E, stamp): old entries precede
//     new ones of equal energy (they arrived earlier), new ones are ordered by candidate
//     index c (the order of the Alg. 3 loop). Slots of evicted entries are reused.
#include "qis_block.cuh"

namespace qis {

constexpr int kMergeThreads = 256;
// kept candidates held in shared memory: min(next_pow2(max(cap, 256)), P.merge_cand), where
// merge_cand is 512 (QIS_MERGE_SMEM_CAND, a power of two in [32, 512], lowers it: a test uses
// it to run the global-memory path)
__host__ __device__ inline int merge_smem_cand(int cap, int merge_cand) {
  const int pc = next_pow2(cap > kMergeThreads ? cap : kMergeThreads);
  return pc < merge_cand ? pc : merge_cand;
}

__global__ void __launch_bounds__(kMergeThreads, 8) k_merge(DevPtrs P) {
  const int b = blockIdx.x;
  const int K1 = P.K1;
  const int lane = threadIdx.x & 31;
  const long long base = (long long)b * K1;
  // every load that depends only on b is issued before any of them is used (one round trip):
  // the active flag, the descriptor, the survivor count, the first survivor entry of this
  // thread (bounded by the capacity, used if below the count), and below the list and the
  // parent
  const int act = P.active[b];
  const InstDesc d = P.inst[b / P.R];
  const int S = P.surv_cnt[b];
  const unsigned long long* sv = P.surv + (long long)b * P.cap;
  const unsigned long long sv0 = ((int)threadIdx.x < P.cap) ? sv[threadIdx.x] : 0ull;
  if (!act) return;
  const int W = d.W;
  if (S > P.cap) {
    if (threadIdx.x == 0) atomicOr(P.status, kStatCapacity);
    return;
  }
  if (threadIdx.x == 0 && S) atomicAdd(P.surv_tot + (b & 63), (unsigned long long)S);
  // kept candidates (key, entry): in shared memory for up to kMergeSmemCand of them (the usual
  // case; a small footprint keeps eight blocks per SM), else in the search's global scratch
  const int PCs = merge_smem_cand(P.cap, P.merge_cand);
  const bool big = S > PCs;
  const int HT = next_pow2(2 * K1);
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long* okey = reinterpret_cast<unsigned long long*>(smem);   // [K1]
  unsigned long long* sk = okey + K1;                                       // [PCs] keys of valid candidates
  unsigned long long* se = sk + PCs;                                        // [PCs] their survivor entries
  if (big) {
    const long long stride = next_pow2(max(P.cap, kMergeThreads));
    sk = P.mrg_scratch + (long long)b * 2 * stride;
    se = sk + stride;
  }
  unsigned long long* sk2 = okey + K1 + 2 * PCs;                            // [kMergeThreads] sorted keys
  unsigned long long* se2 = sk2 + kMergeThreads;                            // [kMergeThreads] sorted entries
  int* oslot = reinterpret_cast<int*>(se2 + kMergeThreads);                 // [K1] slot of old rank r
  uint32_t* htab = reinterpret_cast<uint32_t*>(oslot + K1);                // [HT] duplicate candidates
  __shared__ uint64_t pb[kMaxN / 64];
  __shared__ int s_nv, s_ocut, wsum[33];
  __shared__ unsigned long long s_kmin, s_kmax;
  const bool fp64 = P.mode == QIS_FP64;
  // every load that depends only on b is issued before the first barrier: list length, the key
  // of the last kept entry (T), the parent, the old list's order and keys, and the candidate
  // indices of the kept states one or two flips from the parent (from k_bound: the only
  // candidates that can equal a kept state; one per thread here, any further ones below)
  const int cnt = P.lst_count[b];
  const unsigned long long kT = P.lst_key[base + K1 - 1];   // meaningful when cnt == K1
  const double Ep = fp64 ? P.par_E[b] : 0.0;
  const long long Epq = fp64 ? 0 : P.par_q[b];
  const uint64_t ph = P.par_hash[b];
  const int ndup = P.dup_n[b];
  const uint32_t dc0 = (threadIdx.x < K1) ? P.dup_c[base + threadIdx.x] : kNoCand;
  for (int w = threadIdx.x; w < P.Wmax; w += blockDim.x) pb[w] = P.par_bits[(long long)b * P.Wmax + w];
  for (int r = threadIdx.x; r < K1; r += blockDim.x) {   // two independent coalesced loads
    oslot[r] = P.lst_ord[base + r];
    okey[r] = P.lst_key[base + r];
  }
  for (int k = threadIdx.x; k < HT; k += blockDim.x) htab[k] = kNoCand;
  if (threadIdx.x == 0) {
    s_nv = 0;
    s_ocut = cnt;
    s_kmin = ~0ull;
    s_kmax = 0;
  }
  // threshold: FP64 values in the plain form, exact integers E 2^q otherwise (rank-ordered keys)
  const double T = (cnt == K1 && fp64) ? dkey_inv(kT) : INFINITY;
  const long long Tq = (cnt == K1 && !fp64) ? (long long)(kT ^ (1ull << 63)) : LLONG_MAX;
  // exact energy of survivor t and the threshold test E' < T (strict, Alg. 2); the candidate
  // index c (Sec. III flip order) goes into the entry's low bits. Reads the parent's spins from
  // global memory, so the first block of survivors is evaluated before the first barrier.
  const uint64_t* pbg = P.par_bits + (long long)b * P.Wmax;
  const long long* aqb = fp64 ? nullptr : aq_of(P, b, P.iter_t[b]);
  auto eval = [&](int t, unsigned long long& kk, unsigned long long& ent) -> bool {
    ent = (t == (int)threadIdx.x) ? sv0 : sv[t];
    int i, j;
    surv_sites(ent, i, j);
    ent |= (j < 0) ? (uint32_t)i : pair_index(d.n, i, j);
    const int si = sigma_of(pbg, i), sj = (j >= 0) ? sigma_of(pbg, j) : 0;
    if (fp64) {
      const double* a = P.a64 + (long long)b * P.NP;
      const double de = (j < 0) ? a[i] : dE64(a[i], a[j], P.J64[d.off_mat + (long long)i * d.n_pad + j], si ^ sj);
      const double e = __dadd_rn(Ep, de);
      kk = dkey(e);
      return e < T;
    }
    long long de = aqb[i];
    if (j >= 0) {
      const long long jq = P.Jq[d.off_mat + (long long)i * d.n_pad + j];
      de += aqb[j] + ((si ^ sj) ? -4 * jq : 4 * jq);
    }
    const long long eq = Epq + de;
    kk = qkey(eq);
    return eq < Tq;
  };
  unsigned long long kk0 = 0, ent0 = 0;
  const bool keep0 = (int)threadIdx.x < S && eval(threadIdx.x, kk0, ent0);
  __syncthreads();
  for (int r = threadIdx.x; r < ndup; r += blockDim.x) {
    const uint32_t c = (r == (int)threadIdx.x) ? dc0 : P.dup_c[base + r];
    uint32_t pos = chash(c) & (HT - 1);
    while (atomicCAS(&htab[pos], kNoCand, c) != kNoCand) pos = (pos + 1) & (HT - 1);
  }
  __syncthreads();
  // ---- 1. keep the survivors with E' < T that are not a kept state (the binary search of
  //         Alg. 2: membership of the candidate index among those of the near kept states);
  //         compact the kept ones (warp-aggregated)
  unsigned long long kmn = ~0ull, kmx = 0;   // range of this thread's kept keys
  for (int t0 = 0; t0 < S; t0 += blockDim.x) {
    const int t = t0 + threadIdx.x;
    bool keep = false;
    unsigned long long kk = 0, ent = 0;
    if (t0 == 0) {
      keep = keep0;
      kk = kk0;
      ent = ent0;
    } else if (t < S) {
      keep = eval(t, kk, ent);
    }
    if (keep) {
      const uint32_t c = (uint32_t)ent;
      for (uint32_t pos = chash(c) & (HT - 1); htab[pos] != kNoCand; pos = (pos + 1) & (HT - 1))
        if (htab[pos] == c) {
          keep = false;   // duplicate of a kept state
          break;
        }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (bal) {
      int wb = 0;
      if (lane == 0) wb = atomicAdd(&s_nv, __popc(bal));
      wb = __shfl_sync(0xffffffffu, wb, 0);
      if (keep) {
        const int slot = wb + __popc(bal & ((1u << lane) - 1));
        sk[slot] = kk;          // slot < S <= the buffer's size
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
  // ---- 1b. more than one block of candidates: only the K+1 lowest of them can enter the list
  //          (each later one has K+1 new states below it), so keep the keys up to the (K+1)-th
  //          smallest (ties included) before sorting; compaction in place, chunk by chunk
  if (nv > (int)blockDim.x && nv > K1) {
    __shared__ int hist[256];
    const unsigned long long x = radix_select<unsigned long long>(sk, nv, K1 - 1, hist);
    int kept = 0;
    for (int t0 = 0; t0 < nv; t0 += blockDim.x) {
      const int t = t0 + threadIdx.x;
      unsigned long long kk = 0, ee = 0;
      bool keep = false;
      if (t < nv) {
        kk = sk[t];
        ee = se[t];
        keep = kk <= x;
      }
      int total;
      const int pos = kept + block_exclusive_sum(keep ? 1 : 0, wsum, &total);   // syncs: reads done
      if (keep) {
        sk[pos] = kk;   // pos <= t: never a slot still to be read
        se[pos] = ee;
      }
      kept += total;
      __syncthreads();
    }
    nv = kept;
  }
  // ---- 2. order the kept candidates by (E, c). When the kept keys span less than 2^(64-cb)
  //         (cb = bits of the largest candidate index) one 64-bit value (key - kmin) << cb | c
  //         carries that order: a single-key sort (the usual case)
  const unsigned long long kmin = s_kmin;
  const uint32_t n_cand = (uint32_t)d.n + (uint32_t)((long long)d.n * (d.n - 1) / 2);
  const int cb = 32 - __clz((int)n_cand);   // c <= n_cand - 1 < 2^cb - 1
  const bool packed = nv > 1 && nv <= (int)blockDim.x && ((s_kmax - kmin) >> (64 - cb)) == 0;
  if (packed) {
    sort_runs_packed(sk, se, nv, kmin, cb, sk2);
    sk = sk2;
  } else if (nv > 1) {
    if (nv <= (int)blockDim.x) {
      sort_runs(sk, se, nv, sk2, se2);
      sk = sk2;
      se = se2;
    } else {
      const int m2 = next_pow2(nv);
      for (int t = nv + threadIdx.x; t < m2; t += blockDim.x) {
        sk[t] = ~0ull;
        se[t] = ~0ull;
      }
      __syncthreads();
      bitonic_sort_smem(sk, se, m2);
    }
  }
  __syncthreads();
  // ---- 3. merge with the old list: old entry o -> rank o + #(new with E < E_o) (old entries
  //         precede new ones of equal energy); new entry p -> p + #(old with E <= E_p). Both
  //         ranks grow along their lists, so the evicted old entries (rank >= K+1) are a
  //         suffix o >= s_ocut and the kept new entries a prefix p < K+1 - s_ocut.
  const unsigned long long cmask = (1ull << cb) - 1;
  auto new_key = [&](int p) { return packed ? (sk[p] >> cb) + kmin : sk[p]; };
  for (int o = threadIdx.x; o < cnt; o += blockDim.x) {
    const unsigned long long ko = okey[o];
    int lo = 0, hi = nv;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (new_key(mid) < ko) lo = mid + 1; else hi = mid;
    }
    const int rank = o + lo;
    if (rank < K1) {
      P.lst_ord[base + rank] = oslot[o];
      P.lst_key[base + rank] = ko;
    } else {
      atomicMin(&s_ocut, o);
    }
  }
  __syncthreads();
  // slots for the kept new entries, in order: those of the evicted old entries, then the ones
  // a list that is not yet full has never used (its used slots are 0 .. cnt-1)
  const int ocut = s_ocut, n_ev = cnt - ocut;
  const int t_now = P.iter_t[b];
  for (int p = threadIdx.x; p < nv; p += blockDim.x) {
    const unsigned long long kp = new_key(p);
    int lo = 0, hi = cnt;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (okey[mid] <= kp) lo = mid + 1; else hi = mid;
    }
    const int rank = p + lo;
    if (rank >= K1) continue;
    const int slot = (p < n_ev) ? oslot[ocut + p] : cnt + (p - n_ev);
    uint32_t c;
    int i, j;
    if (packed) {
      c = (uint32_t)(sk[p] & cmask);
      decode_candidate(d.n, c, i, j);
    } else {
      surv_decode(se[p], c, i, j);
    }
    uint64_t* dst = P.lst_bits + (base + slot) * P.Wmax;
    for (int x = 0; x < W; ++x) dst[x] = pb[x] ^ flip_mask(x, i, j);
    if (fp64) {
      P.lst_E[base + slot] = dkey_inv(kp);
    } else {
      // the exact integer E 2^q only: its FP64 value is formed where it is read (the final
      // merge, the host), not once per new entry on the narrow FP64 pipe
      P.lst_q[base + slot] = (long long)(kp ^ (1ull << 63));
    }
    P.lst_stamp[base + slot] = ((uint64_t)t_now << 32) | c;
    P.lst_hash[base + slot] = ph ^ P.zob[i] ^ ((j >= 0) ? P.zob[j] : 0ull);
    P.lst_used[base + slot] = 0;
    P.lst_ord[base + rank] = slot;
    P.lst_key[base + rank] = kp;
  }
  if (threadIdx.x == 0) P.lst_count[b] = min(K1, cnt + nv);
}

size_t merge_smem(int K1, int cap, int merge_cand) {
  const int PCs = merge_smem_cand(cap, merge_cand), HT = next_pow2(2 * K1);
  return (size_t)K1 * 8 + (size_t)PCs * 16 + (size_t)kMergeThreads * 16 + (size_t)K1 * 4 + (size_t)HT * 4;
}

cudaError_t launch_merge(const DevPtrs& P, cudaStream_t s) {
  const size_t sm = merge_smem(P.K1, P.cap, P.merge_cand);
  static size_t attr = 0;
  if (attr < sm) {
    cudaError_t e = cudaFuncSetAttribute(k_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr = sm;
  }
  k_merge<<<P.B, kMergeThreads, sm, s>>>(P);
  return cudaGetLastError();
}

}  // namespace qis
