// qis_final.cu -- Alg. 4: merge of the R kept lists of every instance.
#include "qis_block.cuh"

namespace qis {

// ---------------------------------------------------------------- Alg. 4 merge
// One block per instance. Search 0's list seeds the merged list; the lists of searches
// 1..R-1 are merged in turn. An incoming state already present is skipped (its first
// occurrence wins); the rest are ranked by (E, search, position) and the first K+1 kept.
// Both lists are in ascending E. An incoming entry finds the merged entries of its energy by
// binary search (in the split modes energies are exact, so the copies of a state have equal
// energies; in FP64 they may differ in the last bits, and the entry is compared with every
// merged one), and its rank is its place among the kept incoming entries (a block prefix sum)
// plus the merged entries at or below its energy; a merged entry's rank is its place plus the
// kept incoming entries strictly below it.
struct MergeSet {
  double* E;                // energy
  unsigned long long* S;    // source: search << 32 | position in its list
  uint64_t* H;              // Zobrist hash
  int* R;                   // ref = b * K1 + slot
};

// Set k (0, 1, 2) of the three lists in dynamic shared memory: the 8-byte arrays of all three
// first, then the 4-byte ones (every array aligned for any K1).
__device__ inline MergeSet merge_set(unsigned char* base, int K1, int k) {
  MergeSet m;
  m.E = reinterpret_cast<double*>(base) + (long long)k * K1;
  m.S = reinterpret_cast<unsigned long long*>(base + (size_t)3 * K1 * 8) + (long long)k * K1;
  m.H = reinterpret_cast<uint64_t*>(base + (size_t)6 * K1 * 8) + (long long)k * K1;
  m.R = reinterpret_cast<int*>(base + (size_t)9 * K1 * 8) + (long long)k * K1;
  return m;
}

__device__ inline void merge_put(const MergeSet& to, int t, const MergeSet& from, int f) {
  to.E[t] = from.E[f];
  to.S[t] = from.S[f];
  to.H[t] = from.H[f];
  to.R[t] = from.R[f];
}

__device__ inline bool same_state(const DevPtrs& P, int ra, int rb, int W) {
  const uint64_t* x = P.lst_bits + (long long)ra * P.Wmax;
  const uint64_t* y = P.lst_bits + (long long)rb * P.Wmax;
  for (int w = 0; w < W; ++w)
    if (x[w] != y[w]) return false;
  return true;
}

// first index in v[0..cnt) with v[idx] >= x (strict = false) or v[idx] > x (strict = true)
__device__ inline int bound_of(const double* v, int cnt, double x, bool strict) {
  int lo = 0, hi = cnt;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (strict ? (v[mid] <= x) : (v[mid] < x)) lo = mid + 1; else hi = mid;
  }
  return lo;
}

constexpr int kSetBytes = 8 + 8 + 8 + 4;

__global__ void __launch_bounds__(256) k_final_merge(DevPtrs P) {
  const int inst = blockIdx.x;
  const InstDesc d = P.inst[inst];
  const int K1 = P.K1, W = d.W;
  extern __shared__ __align__(16) unsigned char smem[];
  MergeSet A = merge_set(smem, K1, 0);        // the merged list so far
  const MergeSet N = merge_set(smem, K1, 1);  // the incoming list
  MergeSet T = merge_set(smem, K1, 2);        // the next merged list
  int* cum = reinterpret_cast<int*>(smem + (size_t)3 * K1 * kSetBytes);   // [K1 + 1] kept incoming before p
  int* lev = cum + K1 + 1;                                         // [K1] merged entries <= E_p, or -1
  __shared__ int s_w[33];
  int acnt = 0;
  for (int r = 0; r < P.R; ++r) {
    const int b = d.first_search + r;
    const long long base = (long long)b * K1;
    const int cnt = P.lst_count[b];
    const MergeSet& D = (r == 0) ? A : N;
    for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
      const int slot = P.lst_ord[base + p];
      // split modes keep the exact integer E 2^q of a state; E = that times 2^-q (exact scaling)
      D.E[p] = (P.mode == QIS_FP64) ? P.lst_E[base + slot] : (double)P.lst_q[base + slot] * d.inv_scale;
      D.H[p] = P.lst_hash[base + slot];
      D.R[p] = (int)(base + slot);
      D.S[p] = ((unsigned long long)r << 32) | (unsigned)p;
    }
    __syncthreads();
    if (r == 0) {
      acnt = cnt;
      continue;
    }
    int m = 0;
    for (int p0 = 0; p0 < cnt; p0 += blockDim.x) {
      const int p = p0 + threadIdx.x;
      int keep = 0, le = 0;
      if (p < cnt) {
        const double x = N.E[p];
        const uint64_t hx = N.H[p];
        bool dup = false;
        if (P.mode == QIS_FP64) {
          for (int a = 0; a < acnt && !dup; ++a) dup = A.H[a] == hx && same_state(P, A.R[a], N.R[p], W);
          le = bound_of(A.E, acnt, x, true);
        } else {
          int a = bound_of(A.E, acnt, x, false);
          for (; a < acnt && A.E[a] == x; ++a)
            if (!dup && A.H[a] == hx) dup = same_state(P, A.R[a], N.R[p], W);
          le = a;
        }
        keep = dup ? 0 : 1;
      }
      int tot;
      const int ex = block_exclusive_sum(keep, s_w, &tot);
      if (p < cnt) {
        cum[p] = m + ex;
        lev[p] = keep ? le : -1;
      }
      m += tot;
    }
    if (threadIdx.x == 0) cum[cnt] = m;
    __syncthreads();
    for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
      if (lev[p] < 0) continue;
      const int rank = cum[p] + lev[p];
      if (rank < K1) merge_put(T, rank, N, p);
    }
    for (int a = threadIdx.x; a < acnt; a += blockDim.x) {
      const int rank = a + cum[bound_of(N.E, cnt, A.E[a], false)];
      if (rank < K1) merge_put(T, rank, A, a);
    }
    __syncthreads();
    acnt = min(K1, acnt + m);
    const MergeSet t = A;
    A = T;
    T = t;
  }
  for (int a = threadIdx.x; a < K1; a += blockDim.x) {
    P.mrg_ref[inst * K1 + a] = (a < acnt) ? A.R[a] : -1;
    P.mrg_src[inst * K1 + a] = (a < acnt) ? A.S[a] : ~0ull;
  }
  if (threadIdx.x == 0) P.mrg_count[inst] = acnt;
}

size_t final_merge_smem(int K1) { return (size_t)3 * K1 * kSetBytes + (size_t)(2 * K1 + 1) * 4; }

cudaError_t launch_final_merge(const DevPtrs& P, cudaStream_t s) {
  const size_t sm = final_merge_smem(P.K1);
  static size_t attr = 0;
  if (attr < sm) {
    const cudaError_t e = cudaFuncSetAttribute(k_final_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr = sm;
  }
  k_final_merge<<<P.n_inst, 256, sm, s>>>(P);
  return cudaGetLastError();
}

}  // namespace qis
