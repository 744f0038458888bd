// qis_scan.cu -- candidate scan of the split / integer precision modes (FP32 filter).
//
// Pair candidates (i, j), i < j, of one parent: dE_ij = a_i + a_j + 4 s_i s_j J_ij (Sec. III,
// energy change from the couplings of the flipped sites). A pair survives the filter when
//     y_ij = a_j + (s_i s_j) 4J~_ij  <=  c_i = thr - a_i
// where k_bound derives thr with its error band (c_i is formed here, in FP32).
//
// Work unit = one block task: 32 consecutive rows i (4 warps x 8 rows) and a chunk of 32*NC
// columns j of one instance, for a group of searches of that instance. Each lane keeps its
// 8 x NC couplings 4J~_ij in registers and reuses them for every search; lane l owns columns
// c0 + 32k + l, so every coupling load is a coalesced 128-byte row segment.
//
// Per search the block needs {a_j, s_j} of the chunk's columns and of its rows and a control
// word; one warp stages them with TMA bulk copies (lane p issues search p's three copies) into
// a ring of kRing slots of kPer searches each (completion counted on the slot's mbarrier). The
// warps do not synchronise with each other: each waits for its next slot, works through its
// searches and releases it; the fourth release refills the slot kRing slots ahead. A warp that
// meets many hits may fall behind the others by up to kRing slots without stalling them.
//
// Per slot a warp first votes which of its 8 rows can hit, four searches per ballot: every
// y_ij of the chunk is at least RD(w - max_j |4J~_ij|) (w: minimum a_j over the chunk's
// 256-column window, from the control word; the row maximum of |4J~| from the coupling
// registers), so rows with c_i below it are skipped whole. For each live row (warp-uniform)
// each lane computes y_ij = fma(+-4J~_ij, s_j, a_j) -- the row spin, taken from a ballot so the
// branch is provably uniform, picks the operand sign -- reduces min_j y_ij with three-input
// minima and compares it with c_i. Pairs that must not be evaluated (j <= i, j >= n) hold NaN
// couplings: the FMA propagates NaN and min ignores it. When a row's minimum passes, the lane
// marks which of its columns pass from the same values, and appends one survivor entry per
// passing pair.
#include "qis_block.cuh"

namespace qis {

__device__ __forceinline__ float min3f(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

template <int NC>
__device__ __forceinline__ float rowmin(const float (&y)[NC]) {
  static_assert(NC >= 1 && NC <= 8, "chunk widths 32 .. 256");
  if constexpr (NC == 1) return y[0];
  else if constexpr (NC == 2) return fminf(y[0], y[1]);
  else if constexpr (NC == 3) return min3f(y[0], y[1], y[2]);
  else if constexpr (NC == 4) return min3f(y[0], y[1], fminf(y[2], y[3]));
  else if constexpr (NC == 5) return min3f(min3f(y[0], y[1], y[2]), y[3], y[4]);
  else if constexpr (NC == 6) return min3f(min3f(y[0], y[1], y[2]), y[3], fminf(y[4], y[5]));
  else if constexpr (NC == 7) return min3f(min3f(y[0], y[1], y[2]), min3f(y[3], y[4], y[5]), y[6]);
  else return min3f(min3f(y[0], y[1], y[2]), min3f(y[3], y[4], y[5]), fminf(y[6], y[7]));
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
  return ok != 0;
}
// 1-D bulk copy global -> shared (TMA); completion is counted in bytes on the mbarrier
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

constexpr int kRing = 2;                      // staging ring depth (power of two)
constexpr int kPer = 8;                       // searches per ring slot (two liveness ballots)
constexpr uint64_t kDrainNs = 2000000000ull;   // bound of the waits for copies already issued: 2 s

// Staging ring of one block: slot u % kRing holds searches kPer u .. kPer u + kPer - 1. full[q]
// completes a phase when the slot's bulk copies have landed; rel[q] counts the warps' releases.
struct __align__(128) ScanRing {
  float2 col[kRing][kPer][256];   // {a_j, s_j} of the chunk's columns
  float2 row[kRing][kPer][32];    // {a_i, s_i} of the block's rows
  float4 ctl[kRing][kPer];        // {thr, active, -, w = min a_j over the chunk's 8-group window}
  uint64_t full[kRing];
  int rel[kRing];
  int issued[kRing];
  int err;
};

// EX: spin exchanges only (the pair (i, j) is a candidate only when s_i != s_j): the column
// values are kept twice, as a_j where s_j = -1 (partners of rows with s_i = +1) and as a_j where
// s_j = +1 (rows with s_i = -1), NaN elsewhere, so same-spin pairs never pass.
template <int NC, bool EX>
__device__ __forceinline__ void scan_task(const DevPtrs& P, const InstDesc& d, int row0, int c0, int g, int RG,
                                          ScanRing& sm) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = d.n, np = d.n_pad, NPs = P.NP, cap = P.cap;
  const int b0 = d.first_search + g * RG;   // searches [g RG, g RG + R) of the instance
  const int R = min(RG, P.R - g * RG);
  const float* J4 = P.J4 + d.off_mat;
  const float qnan = __int_as_float(0x7fc00000);
  const int i0 = row0 + warp * 8;
  // bytes of one slot: the chunk's columns (clipped to the row stride; columns past n hold NaN
  // couplings, so whatever the slot holds there never matters), 32 rows, the control word.
  // All sources are 16-byte aligned: NP is a multiple of 128, c0 and row0 of 32.
  const int cols = min(32 * NC, NPs - c0);
  const int nslots = (R + kPer - 1) / kPer;
  // one warp stages slot iteration u into slot q: lane 0 posts the byte count on the slot's
  // barrier, then lane p issues the three copies of search p
  auto stage = [&](int u, int q) {
    const int ns = min(kPer, R - u * kPer);
    if (lane == 0)
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&sm.full[q])),
                   "r"((uint32_t)(ns * (cols * 8 + 32 * 8 + 16))) : "memory");
    __syncwarp();
    if (lane < ns) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the warps' reads first
      const long long b = b0 + u * kPer + lane;
      bulk_g2s(&sm.col[q][lane][0], P.as32 + b * NPs + c0, (uint32_t)(cols * 8), &sm.full[q]);
      bulk_g2s(&sm.row[q][lane][0], P.as32 + b * NPs + row0, 32 * 8, &sm.full[q]);
      bulk_g2s(&sm.ctl[q][lane], P.sctl + b * (NPs / 32) + (c0 >> 5), 16, &sm.full[q]);
    }
    if (lane == 0) sm.issued[q] += 1;
  };
  if (warp == 0) {
    if (lane == 0) {
      for (int q = 0; q < kRing; ++q) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.full[q])));
        sm.rel[q] = 0;
        sm.issued[q] = 0;
      }
      sm.err = 0;
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    for (int u = 0; u < min(kRing, nslots); ++u) stage(u, u);
  }
  __syncthreads();
  // this lane's couplings 4J~_ij, rows i0..i0+7, columns c0 + 32k + lane (NaN where j <= i or
  // j >= n), reused for every search of the group
  float J[8][NC];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int i = i0 + r;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      const int j = c0 + 32 * k + lane;
      J[r][k] = (i < n && j < n && j > i) ? J4[(long long)i * np + j] : qnan;
    }
  }
  // max |4J~_ij| over the task's columns of the row this lane votes for (row i0 + lane % 8);
  // -inf for a row without pairs here (NaN couplings are ignored by fmaxf)
  float rmax = -INFINITY;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    float m = -INFINITY;
#pragma unroll
    for (int k = 0; k < NC; ++k) m = fmaxf(m, fabsf(J[r][k]));
#pragma unroll
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((lane & 7) == r) rmax = m;
  }
  const uint64_t t0 = gtimer();
  int nlive = 0;   // rows this warp evaluated (statistics)
  for (int u = 0; u < nslots; ++u) {
    const int q = u & (kRing - 1);
    const uint32_t par = (uint32_t)(u / kRing) & 1u;
    // bounded wait for the slot; an error anywhere in the block ends every warp's loop
    bool ready = mbar_try(&sm.full[q], par);
    while (!ready) {
      if (*(volatile int*)&sm.err || gtimer() - t0 > P.wait_ns) break;
      ready = mbar_try(&sm.full[q], par);
    }
    if (!__all_sync(0xffffffffu, ready)) {
      if (lane == 0) {
        atomicOr(&sm.err, 1);
        atomicOr(P.status, kStatTimeout);
      }
      break;
    }
    // the slot's rows that can hit, four searches per ballot: lane l takes search 4h + (l >> 3)
    // and row i0 + (l & 7). y_ij >= RD(w - max_j |4J~_ij|) for every column of the chunk
    // (rounding is monotone; w <= a_j), so a row with c_i = fl32(thr - a_i) below it has no
    // pair under its bound
    const int ns = min(kPer, R - u * kPer);
    unsigned long long live64 = 0, neg64 = 0;   // bit 8p + r: row r of search p live / s_i = -1
    float cv[kPer / 4];
#pragma unroll
    for (int h = 0; h < kPer / 4; ++h) {
      const int p = 4 * h + (lane >> 3);
      const float4 ctl = sm.ctl[q][p];   // slots past ns hold stale values: masked below
      const float2 rv = sm.row[q][p][warp * 8 + (lane & 7)];
      cv[h] = __fsub_rn(ctl.x, rv.x);
      live64 |= (unsigned long long)__ballot_sync(0xffffffffu,
                                                  p < ns && ctl.y != 0.f && cv[h] >= __fsub_rd(ctl.w, rmax))
                << (32 * h);
      neg64 |= (unsigned long long)__ballot_sync(0xffffffffu, rv.y < 0.f) << (32 * h);
    }
    nlive += __popcll(live64);
    while (live64) {   // searches with a live row (uniform)
      const int p = (__ffsll((long long)live64) - 1) >> 3;
      const unsigned live = (unsigned)(live64 >> (8 * p)) & 0xffu;
      const unsigned smask = (unsigned)(neg64 >> (8 * p)) & 0xffu;
      live64 &= ~(0xffull << (8 * p));
      const int s = u * kPer + p;
      const float cp = (p >> 2) ? cv[1] : cv[0];
      // column values: {a_j, s_j}; under exchanges a_j twice, masked by the partner's spin
      // (every valid pair has s_i s_j = -1, so y = a_j - 4J~ and s_j is not needed)
      float aj[NC], sj[EX ? 1 : NC], am[EX ? NC : 1];
      {
#pragma unroll
        for (int k = 0; k < NC; ++k) {
          const float2 v = sm.col[q][p][32 * k + lane];
          if constexpr (EX) {
            aj[k] = (v.y < 0.f) ? v.x : qnan;   // partners of rows with s_i = +1
            am[k] = (v.y > 0.f) ? v.x : qnan;   // partners of rows with s_i = -1
          } else {
            aj[k] = v.x;
            sj[k] = v.y;
          }
        }
      }
      {
        unsigned long long cm = 0;   // exact hits of this lane: bit 8r + k = (row i0 + r, column k)
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          if (!((live >> r) & 1u)) continue;   // uniform
          const float c = __shfl_sync(0xffffffffu, cp, (p & 3) * 8 + r);
          float y[NC];
          if constexpr (EX) {   // fl(a_j - 4J~): the same rounding as the FMA with s_i s_j = -1
            if ((smask >> r) & 1u) {
#pragma unroll
              for (int k = 0; k < NC; ++k) y[k] = __fsub_rn(am[EX ? k : 0], J[r][k]);
            } else {
#pragma unroll
              for (int k = 0; k < NC; ++k) y[k] = __fsub_rn(aj[k], J[r][k]);
            }
          } else if ((smask >> r) & 1u) {
#pragma unroll
            for (int k = 0; k < NC; ++k) y[k] = fmaf(-J[r][k], sj[EX ? 0 : k], aj[k]);
          } else {
#pragma unroll
            for (int k = 0; k < NC; ++k) y[k] = fmaf(J[r][k], sj[EX ? 0 : k], aj[k]);
          }
          if (rowmin<NC>(y) <= c) {   // this lane has a hit in row r: which columns
#pragma unroll
            for (int k = 0; k < NC; ++k)
              if (y[k] <= c) cm |= 1ull << (r * 8 + k);
          }
        }
        if (cm) {   // one survivor entry per passing pair: sites i0 + r, c0 + 32k + lane
          int slot = atomicAdd(P.surv_cnt + b0 + s, __popcll(cm));
          unsigned long long* dst = P.surv + (long long)(b0 + s) * cap;
          const unsigned long long e0 = surv_entry(i0, c0 + lane);
          do {
            const int bit = __ffsll((long long)cm) - 1;
            cm &= cm - 1;
            if (slot < cap) dst[slot] = e0 + ((unsigned long long)(bit >> 3) << 32) + ((unsigned long long)(bit & 7) << (kSurvJ + 5));
            ++slot;
          } while (cm);
        }
      }
    }   // searches of the slot
    __syncwarp();
    int last = 0;   // release the slot; the last of the four warps refills it
    if (lane == 0) {
      __threadfence_block();   // this warp's reads of the slot precede the release
      last = (atomicAdd(&sm.rel[q], 1) & 3) == 3;
      if (last) __threadfence_block();   // and every other warp's precede the refill
    }
    if (__shfl_sync(0xffffffffu, last, 0) && u + kRing < nslots) stage(u + kRing, q);
  }
  if (lane == 0 && nlive) atomicAdd(P.eval_cnt + (blockIdx.x & 63), (unsigned long long)nlive * (32 * NC));
  // after an error, wait (bounded) for every copy the block issued before its shared memory
  // is released; without one, every issued copy has been waited for in the loop
  __syncthreads();
  if (threadIdx.x == 0 && sm.err) {
    for (int q = 0; q < kRing; ++q) {
      if (sm.issued[q] == 0) continue;
      const uint32_t par = (uint32_t)(sm.issued[q] - 1) & 1u;
      const uint64_t t1 = gtimer();
      while (!mbar_try(&sm.full[q], par) && gtimer() - t1 < kDrainNs) {
      }
    }
  }
}

// task.x = instance, task.y = first row of the 32-row block, task.z = first column,
// task.w = NC | (search group << 8); a group is RG consecutive searches of the instance
template <bool EX>
__global__ void __launch_bounds__(128, 5) k_scan_pairs(DevPtrs P, const int4* tasks, int n_tasks, int RG) {
  __shared__ ScanRing sm;
  const int4 w = tasks[blockIdx.x];
  const InstDesc d = P.inst[w.x];
  const int g = w.w >> 8;
  switch (w.w & 0xff) {
    case 8: scan_task<8, EX>(P, d, w.y, w.z, g, RG, sm); break;
    case 7: scan_task<7, EX>(P, d, w.y, w.z, g, RG, sm); break;
    case 6: scan_task<6, EX>(P, d, w.y, w.z, g, RG, sm); break;
    case 5: scan_task<5, EX>(P, d, w.y, w.z, g, RG, sm); break;
    case 4: scan_task<4, EX>(P, d, w.y, w.z, g, RG, sm); break;
    case 3: scan_task<3, EX>(P, d, w.y, w.z, g, RG, sm); break;
    case 2: scan_task<2, EX>(P, d, w.y, w.z, g, RG, sm); break;
    default: scan_task<1, EX>(P, d, w.y, w.z, g, RG, sm); break;
  }
}

cudaError_t launch_scan_pairs(const DevPtrs& P, const int4* tasks, int n_tasks, int RG, cudaStream_t s) {
  if (n_tasks <= 0) return cudaSuccess;
  if (P.flips == QIS_FLIPS_EXCHANGE) k_scan_pairs<true><<<n_tasks, 128, 0, s>>>(P, tasks, n_tasks, RG);
  else k_scan_pairs<false><<<n_tasks, 128, 0, s>>>(P, tasks, n_tasks, RG);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- output-sensitive pair scan
// The same filter decided per search with work proportional to its answer (the pruning of the
// Sec. III dE form). In row i the filter value of pair {i, j} is y_ij = fl(a_j + s_i s_j 4J~_ij)
// and the pair passes when y_ij <= c_i = fl32(thr - a_i); since y_ij >= RD(a_j - rm_i) with
// rm_i = max_j |4J~_ij| (rounding is monotone),
//   - row i can pass a pair only if c_i >= RD(amin - rm_i)  (the live rows), and
//   - only with partners a_j < nextup(c_i) + rm_i <= t_i = RU(nextup(c_i) + rm_i) (FP32,
//     rounded up): no partner of any live row lies at or above B = max_i t_i.
// The columns a_j < B are ordered by a monotone bucket of a_j (kSparseNB equal-width buckets
// over [amin, B), a counting sort), so row i's partners all lie in the buckets up to bucket(t_i):
// that prefix of the column order is row i's list. A pair within the threshold passes the
// test of either of its rows (the band of thr bounds the rounding of both forms, which are
// symmetric in i and j), so both sites are live and each is in the other's list: the pair is
// tested once, in the row whose site comes first in the column order, against the columns
// after it. The survivors are therefore a superset of every pair within the threshold, which
// is all the merge needs (it decides every survivor exactly); pairs the rounding puts on the
// other side of thr in one form or the other may differ from the dense scan's, never a pair
// the merge keeps. No FP64 arithmetic: GB300's FP64 pipe is narrow.
// One block per search: stage {a_j, s_j} and rm_j; list the live rows and B; count, scan and
// scatter the columns by bucket (each site's spin and position packed into its staged s_j);
// each live row's list length from its bucket, less its own position; offsets by a block scan;
// then the flat list of (row, column) pairs, one thread each, their coupling loads issued four
// at a time, survivors appended with one shared atomic per warp. The per-search work is the
// live rows times their lists (several hundred pairs a search for n = 600, K = 120, against
// n(n-1)/2 = 179700), a chain of short dependent steps: the loads it cannot avoid are grouped
// so that each step waits once.
template <bool EX>
__global__ void __launch_bounds__(128, 16) k_scan_sparse(DevPtrs P) {
  constexpr int SB = 5;   // sites staged per thread and pass (n = 600: one pass)
  constexpr int PB = 4;   // listed pairs per thread and pass (their coupling loads issued together)
  const int b = blockIdx.x;
  if (!P.active[b]) return;
  const InstDesc d = P.inst[b / P.R];
  const int n = d.n, NP = P.NP, tid = threadIdx.x, lane = tid & 31;
  const float thr = P.thr32[b], amin = P.amin32[b];
  extern __shared__ float2 sa[];                              // [NP] {a_j, s_j}
  int* li = reinterpret_cast<int*>(sa + NP);                  // [NP] live rows
  int* pc = li + NP;                                          // [NP] rm of each live row, then list offsets
  int* cj = pc + NP;                                          // [NP] columns in bucket order
  __shared__ int s_nl, s_ns, s_w[4], bs[kSparseNB + 1], bcur[kSparseNB];
  __shared__ float wB[4];
  const float2* g = P.as32 + (long long)b * NP;
  const float* rm = P.rm4 + d.off_vec;
  // 1. stage {a, s} (the first pass's loads are issued before the first barrier); live rows
  //    with their rm; B
  float2 v[SB];
  float r[SB];
#pragma unroll
  for (int u = 0; u < SB; ++u) {
    const int i = tid + u * 128;
    if (i < n) {
      v[u] = g[i];
      r[u] = rm[i];
    }
  }
  if (tid == 0) {
    s_nl = 0;
    s_ns = P.surv_cnt[b];   // the singles k_bound listed; this block alone appends to the search
  }
  for (int k = tid; k < kSparseNB; k += 128) bcur[k] = 0;
  __syncthreads();
  float bl = -INFINITY;
  for (int base = 0; base < n; base += SB * 128) {
    if (base > 0) {
#pragma unroll
      for (int u = 0; u < SB; ++u) {
        const int i = base + tid + u * 128;
        if (i < n) {
          v[u] = g[i];
          r[u] = rm[i];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < SB; ++u) {
      const int i = base + tid + u * 128;
      if (i < n) {
        sa[i] = v[u];
        const float c = __fsub_rn(thr, v[u].x);
        if (c >= __fsub_rd(amin, r[u])) {
          const int q = atomicAdd(&s_nl, 1);
          li[q] = i;
          pc[q] = __float_as_int(r[u]);
          bl = fmaxf(bl, __fadd_ru(nextafterf(c, INFINITY), r[u]));   // +inf for c = +inf
        }
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) bl = fmaxf(bl, __shfl_xor_sync(0xffffffffu, bl, o));
  if (lane == 0) wB[tid >> 5] = bl;
  __syncthreads();
  const int nl = s_nl;
  if (nl == 0) return;   // block-uniform
  const float B = fmaxf(fmaxf(wB[0], wB[1]), fmaxf(wB[2], wB[3]));
  // 2. bucket of every column a_j < B: equal widths over [amin, B) (one bucket when that range
  //    is not finite); count, exclusive scan (warp 0), scatter
  const float span = __fsub_ru(B, amin);
  const float inv = (span > 0.f && span < INFINITY) ? __fdiv_rn((float)kSparseNB, span) : 0.f;
  for (int j = tid; j < n; j += 128)
    if (sa[j].x < B) atomicAdd(&bcur[sparse_bucket(sa[j].x, amin, inv)], 1);
  __syncthreads();
  if (tid < 32) {
    int x[kSparseNB / 32], s = 0;
#pragma unroll
    for (int k = 0; k < kSparseNB / 32; ++k) {
      x[k] = bcur[lane * (kSparseNB / 32) + k];
      s += x[k];
    }
    int inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    int acc = inc - s;
#pragma unroll
    for (int k = 0; k < kSparseNB / 32; ++k) {
      bs[lane * (kSparseNB / 32) + k] = acc;
      bcur[lane * (kSparseNB / 32) + k] = acc;
      acc += x[k];
    }
    if (lane == 31) bs[kSparseNB] = acc;
  }
  __syncthreads();
  // site code in place of s_j: (position in the column order << 1) | sigma_j, or INT_MIN |
  // sigma_j for a site at or above B
  for (int j = tid; j < n; j += 128) {
    const float2 v = sa[j];
    const int sg = v.y < 0.f;
    int code = INT_MIN | sg;
    if (v.x < B) {
      const int k = atomicAdd(&bcur[sparse_bucket(v.x, amin, inv)], 1);
      cj[k] = j;
      code = (k << 1) | sg;
    }
    sa[j].y = __int_as_float(code);
  }
  // each live row's list: the buckets up to that of t_i (a_j < t_i gives bucket(a_j) <=
  // bucket(t_i): the bucket is monotone)
  for (int q = tid; q < nl; q += 128) {
    const int i = li[q];
    const float c = __fsub_rn(thr, sa[i].x), rr = __int_as_float(pc[q]);
    pc[q] = bs[sparse_bucket(__fadd_ru(nextafterf(c, INFINITY), rr), amin, inv) + 1];
  }
  __syncthreads();
  // the columns after the row's own position (none for a row outside the column order), then
  // exclusive offsets: each thread a run of consecutive rows, a warp and a block scan
  {
    const int per = (nl + 127) >> 7, q0 = min(nl, tid * per), q1 = min(nl, q0 + per);
    int sum = 0;
    for (int q = q0; q < q1; ++q) {
      const int code = __float_as_int(sa[li[q]].y);
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
    if (lane == 31) s_w[tid >> 5] = inc;
    __syncthreads();
    int acc = inc - sum;
    for (int w = 0; w < (tid >> 5); ++w) acc += s_w[w];
    for (int q = q0; q < q1; ++q) {
      const int x = pc[q];
      pc[q] = acc;
      acc += x;
    }
  }
  __syncthreads();
  // 3. the listed pairs, one thread each, PB at a time; survivors appended with one
  //    shared-memory atomic per warp (one block per search: the count goes back to global
  //    memory once, at the end)
  const int tot = s_w[0] + s_w[1] + s_w[2] + s_w[3], cap = P.cap;
  const float* J4 = P.J4 + d.off_mat;
  unsigned long long* surv = P.surv + (long long)b * cap;
  int nev = 0;
  for (int t0 = 0; t0 < tot; t0 += PB * 128) {   // block-uniform trip count
    float cv[PB], av[PB], pv[PB], jv[PB];
    int ij[PB];
    bool ok[PB];
#pragma unroll
    for (int u = 0; u < PB; ++u) {
      const int t = t0 + u * 128 + tid;
      ok[u] = false;
      if (t < tot) {
        int lo = 0, hi = nl;   // the row q with pc[q] <= t < pc[q + 1]
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (pc[mid] <= t) lo = mid; else hi = mid;
        }
        const int i = li[lo];
        const float2 vi = sa[i];
        const int ci = __float_as_int(vi.y);
        const int j = cj[(ci >> 1) + 1 + t - pc[lo]];
        const float2 vj = sa[j];
        ij[u] = min(i, j) | (max(i, j) << 16);   // n <= 16384
        cv[u] = __fsub_rn(thr, vi.x);
        av[u] = vj.x;
        pv[u] = ((ci ^ __float_as_int(vj.y)) & 1) ? -1.f : 1.f;   // s_i s_j
        ok[u] = !EX || pv[u] < 0.f;   // exchanges: opposite spins only
        if (ok[u]) jv[u] = J4[(long long)i * d.n_pad + j];
      }
    }
#pragma unroll
    for (int u = 0; u < PB; ++u) {
      bool hit = false;
      if (ok[u]) {
        ++nev;
        hit = fmaf(pv[u], jv[u], av[u]) <= cv[u];   // fl(a_j + s_i s_j 4J~_ij) <= c_i
      }
      const unsigned m = __ballot_sync(0xffffffffu, hit);
      if (m) {
        const int leader = __ffs(m) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(&s_ns, __popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        const int slot = base + __popc(m & ((1u << lane) - 1u));
        if (hit && slot < cap) surv[slot] = surv_entry(ij[u] & 0xffff, ij[u] >> 16);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nev += __shfl_xor_sync(0xffffffffu, nev, o);
  if (lane == 0 && nev) atomicAdd(P.eval_cnt + (b & 63), (unsigned long long)nev);
  __syncthreads();
  if (tid == 0) P.surv_cnt[b] = s_ns;
}

size_t scan_sparse_smem(int NP) { return (size_t)NP * 8 + (size_t)NP * 12; }

cudaError_t launch_scan_sparse(const DevPtrs& P, cudaStream_t s) {
  const size_t sm = scan_sparse_smem(P.NP);
  static size_t attr[2] = {0, 0};
  const int ex = P.flips == QIS_FLIPS_EXCHANGE;
  if (attr[ex] < sm) {
    cudaError_t e = ex ? cudaFuncSetAttribute(k_scan_sparse<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)
                       : cudaFuncSetAttribute(k_scan_sparse<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr[ex] = sm;
  }
  if (ex) k_scan_sparse<true><<<P.B, 128, sm, s>>>(P);
  else k_scan_sparse<false><<<P.B, 128, sm, s>>>(P);
  return cudaGetLastError();
}

// Host: cover the pairs (i < j) of an n-spin instance with block tasks. Block a holds rows
// [32a, 32a+32); its w = n - 32a columns (from 32a: the 32 x 32 diagonal block is masked inside
// the task) are split into m = ceil(w / (32 nc_max)) chunks of equal width 32 NC,
// NC = ceil(w / 32m) <= nc_max, so no task is narrow; columns past n are masked. Each chunk is
// repeated for the ceil(R / RG) groups of RG searches.
void scan_tasks_for(int inst, int n, int nc_max, int R, int RG, std::vector<int4>& out) {
  const int groups = (R + RG - 1) / RG;
  for (int row0 = 0; row0 < n - 1; row0 += 32) {
    const int w = n - row0;
    const int m = (w + 32 * nc_max - 1) / (32 * nc_max);
    const int nc = (w + 32 * m - 1) / (32 * m);
    for (int g = 0; g < groups; ++g)
      for (int k = 0; k < m; ++k) out.push_back(make_int4(inst, row0, row0 + 32 * nc * k, nc | (g << 8)));
  }
}

}  // namespace qis
