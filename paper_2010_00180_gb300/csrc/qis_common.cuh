// qis_common.cuh -- types and helpers shared by the CUDA translation units of libqis.
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <vector>

#include "../../include/qis.h"

namespace qis {

constexpr int kTile = 64;        // scan tile edge (sites)
constexpr int kPad = 128;        // n is padded to a multiple of this (tensor-core M tile)
constexpr int kMaxDigits = 5;    // 12-bit signed digits (base 4096) of the fixed-point couplings
constexpr int kMaxN = 16384;
constexpr int kScan64Group = 4;  // searches per block of the FP64 pair scan

// Device error flags (bit mask in ctx status word).
constexpr int kStatCapacity = 1;
constexpr int kStatTimeout = 2;
constexpr int kStatBadParent = 4;

// Per-instance descriptor (device and host copies).
struct InstDesc {
  int n;            // spins
  int n_pad;        // n rounded up to kPad
  int W;            // words per state
  int q;            // fixed-point exponent: Jq = J * 2^q  (-1 in FP64 mode)
  int digits;       // number of balanced base-2^dbits digits of Jq
  int dbits;        // digit width: 12 bits, 11 above n_pad = 8192 (FP32 partial sums of the digit
                    // GEMM stay below 2^24: |digit| <= 2^(dbits-1), n_pad terms)
  int first_search; // global index of search r = 0 of this instance
  long long off_mat;  // element offset of this instance's n_pad x n_pad matrices
  long long off_vec;  // element offset of this instance's n_pad vectors
  double inv_scale;   // 2^-q
  float j4max;        // max |fl32(4 J_ij)|
  double j4max64;    // 4 max |J_ij| (exact in FP64)
  int rounded;        // input was rounded onto the grid
};

// Device pointers of one context (passed to kernels by value).
struct DevPtrs {
  const InstDesc* inst;
  int n_inst, R, K1, Wmax, cap, mode, B;
  int NP;                 // row stride of per-search site arrays (max n_pad)
  int flips;              // QIS_FLIPS_*: the candidate set
  int dense_ctl;          // 1: k_bound writes the dense pair scan's control words (sctl)
  // instance pools
  const double* J64;      // [off_mat + i*n_pad + j]
  const long long* Jq;    // fixed-point couplings
  const float* J4;        // fl32(4 * J)
  const __half* D16;      // digit planes [d][inst][i][NP] (row stride NP), plane = pool_mat elements
  long long pool_mat;     // elements of one digit plane
  const double* h64;      // [off_vec + i]
  const long long* hq;
  const uint64_t* zob;    // Zobrist keys [kMaxN]
  // per-search state, search b
  uint64_t* lst_bits;     // [b][K1][Wmax]
  double* lst_E;          // [b][K1] FP64 mode (and the initial and imported entries); split modes: lst_q
  long long* lst_q;       // [b][K1] exact E * 2^q of each slot (split modes)
  unsigned long long* lst_key;  // [b][K1] order key of the entry of rank r (qkey of E 2^q, or dkey of E)
  uint64_t* lst_stamp;    // [b][K1]
  uint64_t* lst_hash;     // [b][K1]
  uint8_t* lst_used;      // [b][K1]
  int* lst_ord;           // [b][K1] slot of rank r
  int* lst_count;         // [b]
  uint64_t* par_bits;     // [b][Wmax]
  double* par_E;          // [b]
  long long* par_q;       // [b] exact E_p * 2^q (split modes)
  uint64_t* par_hash;     // [b]
  int* active;            // [b]
  int* iter_t;            // [b] iterations done
  long long* aq;          // [ring_n][b][NP] exact a_i * 2^q of the parent of iteration t in slot t % ring_n (split modes)
  int ring_n;             // slots of the aq ring
  long long ring_slot;    // elements of one slot (every search of the context)
  int inc_on;             // local fields by incremental update from the generating parent's (split modes)
  uint64_t* par_stamp;    // [b] stamp (t << 32 | c) of the parent: its generating iteration and flips
  int* ring_t0;           // [b] iterations <= ring_t0 have no aq ring entry (imported lists)
  int* full_tile;         // [inst][ceil(R / gemm_nt)] 1: a search of the tensor-core tile needs full fields
  float2* as32;           // [b][n_pad] {fl32(a_i), s_i} (split modes)
  double* a64;            // [b][n_pad] FP64 a_i (FP64 mode)
  float* thr32;           // [b] scan threshold on dE (split modes)
  float* amin32;          // [b] min_i fl32(a_i) of the parent (split modes; the sparse scan's row bound)
  float* rm4;             // [off_vec + i] max_j |4J~_ij| of row i (split modes, per instance)
  float4* sctl;           // [b][NP/32] scan control word per 32-column group (k_bound)
  double* thrE;           // [b] FP64 mode: E' must be < thrE[b] ...
  double* capE;           // [b] ... and <= capE[b]
  double* amin64;         // [b] FP64 mode: min_i a_i of the parent (the scan's row bound)
  int* surv_cnt;          // [b]
  uint32_t* dup_c;        // [b][K1] candidate index of every kept state one or two flips from the parent
  int* dup_n;             // [b] their number
  unsigned long long* surv;  // [b][cap] survivor entries {i, j} (surv_entry; c filled by the merge)
  int merge_cand;         // kept candidates the merge holds in shared memory (512; power of two)
  unsigned long long* mrg_scratch;  // [b][2][next_pow2(max(cap, 256))] the merge's keys and entries when they exceed shared memory
  __half* S16;            // +-1 spins of the parents (0 past n), tensor-core operand, tiled (s16_offset)
  long long s16_stride;   // halves of one instance's region of S16
  int gemm_nt;            // searches per tensor-core tile (the S16 tiling)
  uint64_t* init_bits;    // [b][Wmax]
  double* init_E;         // [b] energy of the initial state (set with it)
  long long* init_q;      // [b] the same, exact E 2^q (split modes)
  int* e0_pend;           // [b] 1: E(psi0) not formed yet; the fused search kernel's first
                          // iteration forms it from psi0's exact fields (split modes)
  int* status;            // [0] error bits
  unsigned long long wait_ns;  // bound of every device-side wait (%globaltimer ns; 2 s by default)
  int wait_probe;         // 1: the field GEMM's MMA thread first waits on a barrier that nothing
                          // completes (tests the timeout path); 0 otherwise
  int* nprod;             // [b] productive iterations (a parent was expanded) of search b
  unsigned long long* npair;  // [b] pair candidates of the expanded parents of search b
  unsigned long long* eval_cnt;  // [64] pair terms the FP32 scan evaluated (live rows x chunk width)
  unsigned long long* surv_tot;  // [64] survivors the merge read (sum of the per-search counts)
  // final merge (Alg. 4) per instance
  int* mrg_ref;           // [inst][K1] search*K1 + slot
  uint64_t* mrg_src;      // [inst][K1]
  int* mrg_count;         // [inst]
  // rescoring from scratch: partial sums (sum of J over differing spins, sum of all J; int64 or
  // FP64) per output state and row part when the rows of a group of states are split over blocks
  unsigned long long* rs_acc;   // [states][32][2]
  int sms;                      // streaming multiprocessors of the device
};

__host__ __device__ inline int words_of(int n) { return (n + 63) >> 6; }

// aq of search b at iteration t (the ring slot of that iteration's parent)
__host__ __device__ inline long long* aq_of(const DevPtrs& P, long long b, int t) {
  return P.aq + (long long)(t % P.ring_n) * P.ring_slot + b * P.NP;
}

// Tensor-core operands are stored pre-tiled in the exact shared-memory image of a K-major
// operand with 128-byte swizzle: a tile is rows x 64 FP16 (128 bytes per row), 8-row groups
// of 1024 bytes, and the 16-byte chunk c of row r sits at chunk c ^ (r & 7). One contiguous bulk
// copy then moves a whole tile into place.
__host__ __device__ inline long long swz_in_tile(int r, int k) {
  return (long long)r * 64 + ((((k & 63) >> 3) ^ (r & 7)) << 3) + (k & 7);
}
// Element (i, j) of one instance's digit plane: 128 x 64 tiles, row-block major.
__host__ __device__ inline long long d16_offset(int i, int j, int NP) {
  return ((long long)(i >> 7) * (NP >> 6) + (j >> 6)) * 8192 + swz_in_tile(i & 127, j);
}
// Spin k of search r (0 <= r < R) of one instance's S16 region: NT x 64 tiles, tile block of
// searches major.
__host__ __device__ inline long long s16_offset(int r, int k, int NT, int NP) {
  return ((long long)(r / NT) * (NP >> 6) + (k >> 6)) * ((long long)NT * 64) + swz_in_tile(r % NT, k);
}
__host__ __device__ inline int pad_of(int n) { return (n + kPad - 1) / kPad * kPad; }

// candidate index <-> sites: c < n single i = c; c >= n pair (i, j), i < j, lexicographic
__host__ __device__ inline uint32_t pair_index(int n, int i, int j) {
  return (uint32_t)n + (uint32_t)((long long)i * n - (long long)i * (i + 1) / 2 + (j - i - 1));
}
// Survivor entry: bits 32-45 site i, bits 46-59 site j, bit 60 set for a single flip (no j);
// n <= 16384 keeps i and j in 14 bits. The candidate filters (singles by k_bound, pairs by the
// scans) write the sites only; the merge fills bits 0-31 with the candidate index c (the
// tie-break of equal energies) when it reads the entry.
constexpr int kSurvJ = 46;   // bit position of site j
__host__ __device__ inline unsigned long long surv_entry(int i, int j) {
  return ((unsigned long long)(unsigned)i << 32) |
         (j < 0 ? (1ull << 60) : ((unsigned long long)(unsigned)j << kSurvJ));
}
__host__ __device__ inline void surv_sites(unsigned long long e, int& i, int& j) {
  i = (int)((e >> 32) & 0x3fffu);
  j = ((e >> 60) & 1u) ? -1 : (int)((e >> kSurvJ) & 0x3fffu);
}
__host__ __device__ inline void surv_decode(unsigned long long e, uint32_t& c, int& i, int& j) {
  c = (uint32_t)e;
  surv_sites(e, i, j);
}

__device__ inline void decode_candidate(int n, uint32_t c, int& i, int& j) {
  if (c < (uint32_t)n) { i = (int)c; j = -1; return; }
  long long r = (long long)c - n;
  // row i holds n-1-i pairs; start(i) = i*n - i*(i+1)/2. The closed form in FP32 lands within
  // a step or two of the row (r < 2^23); the integer loops below make it exact. (FP64 here
  // would cost every thread a double square root on GB300's narrow FP64 pipe.)
  const float nn = 2.f * n - 1.f;
  int ii = (int)((nn - sqrtf(fmaxf(nn * nn - 8.f * (float)r, 0.f))) * 0.5f);
  if (ii < 0) ii = 0;
  if (ii > n - 2) ii = n - 2;
  while (ii > 0 && (long long)ii * n - (long long)ii * (ii + 1) / 2 > r) --ii;
  while (ii < n - 2 && (long long)(ii + 1) * n - (long long)(ii + 1) * (ii + 2) / 2 <= r) ++ii;
  i = ii;
  j = (int)(r - ((long long)ii * n - (long long)ii * (ii + 1) / 2)) + ii + 1;
}

__device__ inline int sigma_of(const uint64_t* bits, int i) { return (int)((bits[i >> 6] >> (i & 63)) & 1ull); }

// SplitMix64 (Steele, Lea and Flood 2014): value number c of the stream started at key.
__host__ __device__ inline uint64_t splitmix64(uint64_t key, uint64_t c) {
  uint64_t z = key + (c + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// orderable 64-bit key of a double (ascending doubles -> ascending unsigned)
__device__ inline unsigned long long dkey(double x) {
  x = x + 0.0;  // -0.0 -> +0.0
  unsigned long long u = (unsigned long long)__double_as_longlong(x);
  return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}

// order-preserving key of an exact integer energy E 2^q (signed -> unsigned)
__host__ __device__ inline unsigned long long qkey(long long x) { return (unsigned long long)x ^ (1ull << 63); }

__host__ __device__ inline int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// FP64 energy change of the pair flip (i, j): (a_i + a_j) + 4 s_i s_j J_ij, the product exact
__device__ inline double dE64(double ai, double aj, double j, int flip) {
  return __dadd_rn(__dadd_rn(ai, aj), flip ? -4.0 * j : 4.0 * j);
}

__device__ inline double dkey_inv(unsigned long long k) {
  return __longlong_as_double((long long)((k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k));
}

// Warp-parallel search of a 256-bin histogram: the bin holding the rank-th element (0-based),
// and the rank of that element within the bin. Called by one full warp.
__device__ inline void find_bin(const int* hist, int rank, int& bin, int& within) {
  const int lane = threadIdx.x & 31;
  int loc[8], s = 0;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    loc[u] = hist[lane * 8 + u];
    s += loc[u];
  }
  int incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const unsigned m = __ballot_sync(0xffffffffu, incl > rank);
  const int L = m ? __ffs(m) - 1 : 31;
  int r = rank - __shfl_sync(0xffffffffu, incl - s, L);
  int bb = 255;
  if (lane == L) {
    int u = 0;
    for (; u < 7; ++u) {
      if (r < loc[u]) break;
      r -= loc[u];
    }
    bb = L * 8 + u;
  }
  bin = __shfl_sync(0xffffffffu, bb, L);
  within = __shfl_sync(0xffffffffu, r, L);
}

// Block-wide radix select: the rank-th smallest (0-based) of `cnt` keys in smem, 8 bits per
// pass from the top. `hist` holds 256 counters. Every thread of the block must call it.
template <typename K>
__device__ K radix_select(const K* keys, int cnt, int rank, int* hist) {
  __shared__ K s_prefix;
  __shared__ int s_rank;
  K prefix = 0, mask = 0;
  constexpr int kBits = 8 * sizeof(K);
  for (int shift = kBits - 8; shift >= 0; shift -= 8) {
    for (int t = threadIdx.x; t < 256; t += blockDim.x) hist[t] = 0;
    __syncthreads();
    // warp-aggregated: the lanes of a warp that fall into one bin add once (most keys share
    // their leading bits, so plain atomics would serialise on one counter)
    for (int t0 = 0; t0 < cnt; t0 += blockDim.x) {
      const int t = t0 + threadIdx.x;
      const bool in = t < cnt && (keys[t] & mask) == prefix;
      const unsigned act = __ballot_sync(0xffffffffu, in);
      if (in) {
        const int bin = (int)((keys[t] >> shift) & 255);
        const unsigned peers = __match_any_sync(act, bin);
        if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&hist[bin], __popc(peers));
      }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      int dgt, r;
      find_bin(hist, rank, dgt, r);
      if (threadIdx.x == 0) {
        s_prefix = prefix | ((K)dgt << shift);
        s_rank = r;
      }
    }
    __syncthreads();
    prefix = s_prefix;
    rank = s_rank;
    mask |= (K)255 << shift;
    __syncthreads();
  }
  return prefix;
}

// Message returned by qis_last_error(NULL) (calls that have no context).
void set_global_error(const char* msg);

// Learned warm start (qis_mlp.cu): R initial states of one instance into init_bits.
cudaError_t mlp_propose_states(qis_mlp* m, const double* J64, long long stride, const double* h64, int n, int R,
                               uint64_t key, uint64_t* init_bits, int Wstride, cudaStream_t s);
int mlp_max_n(const qis_mlp* m);

// Kernel launchers (defined in the .cu files); each returns the cudaError_t of the launch.
cudaError_t launch_restride(const double* src, int n, int n_pad, double* dst, cudaStream_t s);
// Where one instance of a creation batch was staged and where its layout and statistics go.
struct LayoutItem {
  const double* src;   // n x n FP64, contiguous, as copied from the host
  long long off_mat, off_vec;
  int n, n_pad;
  double* stats;       // its validation statistics (NP + 8 doubles)
};
cudaError_t launch_layout_batch(const DevPtrs& P, const LayoutItem* items, int count, int max_n_pad, double* J64,
                                cudaStream_t s);
cudaError_t launch_prepare_batch(const DevPtrs& P, int first, int count, int max_n_pad, __half* D16, long long* Jq,
                                 float* J4, long long* hq, cudaStream_t s);
cudaError_t launch_rowmax4(const DevPtrs& P, const InstDesc& d, cudaStream_t s);
cudaError_t launch_scan_sparse(const DevPtrs& P, cudaStream_t s);
constexpr int kSparseMaxNP = 4096;   // the sparse pair scan's largest padded n (shared-memory lists)
// The fused search kernel (every iteration of a search in one block): its largest padded n and
// list length (per-search arrays in shared memory).
constexpr int kSearchMaxNP = 1024;
constexpr int kSearchMaxK1 = 256;
cudaError_t launch_search(const DevPtrs& P, int n_iters, cudaStream_t s);
size_t search_smem(const DevPtrs& P);
cudaError_t launch_validate(const DevPtrs& P, int inst, int n, long long off_mat, long long off_vec,
                            double* stats, cudaStream_t s);
cudaError_t launch_fields_tc(const DevPtrs& P, const void* D16, const void* S16, int max_inst, int digits_max,
                             int nt, cudaStream_t s);
int gemm_tile_n(int R, int digits);
cudaError_t launch_quantize(const DevPtrs& P, const InstDesc& d, int inst, __half* D16, long long* Jq,
                            float* J4, long long* hq, cudaStream_t s);
cudaError_t launch_init_search(const DevPtrs& P, int b0, int nb, cudaStream_t s, bool cached = false,
                               bool deferred = false);
cudaError_t launch_hash_list(const DevPtrs& P, int b, int count, cudaStream_t s);
cudaError_t launch_pick(const DevPtrs& P, cudaStream_t s);
cudaError_t launch_fields_exact(const DevPtrs& P, cudaStream_t s);
cudaError_t launch_fields_inc(const DevPtrs& P, cudaStream_t s);
cudaError_t launch_fields_fp64(const DevPtrs& P, cudaStream_t s);
cudaError_t launch_bound(const DevPtrs& P, cudaStream_t s);
cudaError_t launch_scan_pairs(const DevPtrs& P, const int4* tasks, int n_tasks, int RG, cudaStream_t s);
cudaError_t launch_scan64(const DevPtrs& P, const int4* work, int n_work, cudaStream_t s);
void scan_tasks_for(int inst, int n, int nc_max, int R, int RG, std::vector<int4>& out);
cudaError_t launch_merge(const DevPtrs& P, cudaStream_t s);
cudaError_t launch_final_merge(const DevPtrs& P, cudaStream_t s);
size_t merge_smem(int K1, int cap, int merge_cand);
size_t final_merge_smem(int K1);
cudaError_t launch_rescore(const DevPtrs& P, const InstDesc& d, const uint64_t* bits, int count, int Wn,
                           double* E_out, cudaStream_t s);
cudaError_t launch_topk_all(const DevPtrs& P, int k, bool all_exact, int max_n, uint64_t* out, double* E,
                            cudaStream_t s);
cudaError_t launch_init_energy(const DevPtrs& P, int inst0, int n_inst, int max_n, cudaStream_t s);
cudaError_t launch_gather_merged(const DevPtrs& P, int inst, const InstDesc& d, int k, uint64_t* bits_out,
                                 cudaStream_t s);

}  // namespace qis
