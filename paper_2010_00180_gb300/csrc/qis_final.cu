// qis_final.cu -- Alg. 4: merge of the R kept lists of every instance.
#include "qis_common.cuh"

namespace qis {

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
      // split modes keep the exact integer E 2^q of a state; E = that times 2^-q (exact scaling)
      nE[p] = (P.mode == QIS_FP64) ? P.lst_E[base + slot] : (double)P.lst_q[base + slot] * d.inv_scale;
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
