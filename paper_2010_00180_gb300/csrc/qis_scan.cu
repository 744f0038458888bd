// qis_scan.cu -- candidate scan of the split / integer precision modes (FP32 filter).
//
// Pair candidates (i, j), i < j, of one parent: dE_ij = a_i + a_j + 4 s_i s_j J_ij (Sec. III,
// energy change from the couplings of the flipped sites). A pair survives the filter when
//     y_ij = a_j + (s_i s_j) 4J~_ij  <=  c_i = thr - a_i
// where k_bound derives thr with its error band and writes c_i per site.
//
// Work unit = one block task: 32 consecutive rows i (4 warps x 8 rows) and a chunk of 32*NC
// columns j of one instance, for all R searches of that instance. Each lane keeps its 8 x NC
// couplings 4J~_ij in registers and reuses them for every search; lane l owns columns
// c0 + 32k + l, so every coupling load is a coalesced 128-byte row segment. Per search the
// block stages {a_j, s_j} of the chunk's columns, {c_i, s_i} of its rows and {thr, active} with
// cp.async, two searches ahead (triple buffer, one block barrier per search).
//
// Per search and row (warp-uniform) each lane computes y_ij = fma(+-4J~_ij, s_j, a_j) -- the
// row spin, taken from a ballot so the branch is provably uniform, picks the operand sign --
// reduces min_j y_ij with three-input minima and compares it with c_i. Pairs that must not be
// evaluated (j <= i, j >= n) hold NaN couplings: the FMA propagates NaN and min ignores it.
// A lane whose rows hit appends one record {rows, its columns, row mask}; the merge expands it
// with the same FP32 test, so the filter decision is identical in both places.
#include "qis_common.cuh"

namespace qis {

constexpr int kBufs = 3;   // staging depth: search s is computed while s+1, s+2 land

__device__ __forceinline__ float min3f(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

template <int NC>
__device__ __forceinline__ float rowmin(const float (&y)[NC]) {
  if constexpr (NC == 1) {
    return y[0];
  } else if constexpr (NC == 2) {
    return fminf(y[0], y[1]);
  } else if constexpr (NC == 4) {
    return min3f(y[0], y[1], fminf(y[2], y[3]));
  } else {
    static_assert(NC == 8, "chunk widths 32, 64, 128, 256");
    return min3f(min3f(y[0], y[1], y[2]), min3f(y[3], y[4], y[5]), fminf(y[6], y[7]));
  }
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  const int sz = valid ? 16 : 0;   // 0 bytes read -> 16 zero bytes written
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(sz) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Record layout of a scan hit (bit 63 set): bits 0-15 first of the lane's 8 rows, bits 16-31
// the lane's first column jb (its columns are jb + 32k, k < NC), bits 32-36 NC, bits 37-44
// mask of the rows that hit.
__host__ __device__ inline unsigned long long make_record(int i0, int jb, int nc, unsigned hm) {
  return (1ull << 63) | (unsigned long long)(unsigned)i0 | ((unsigned long long)(unsigned)jb << 16) |
         ((unsigned long long)(unsigned)nc << 32) | ((unsigned long long)(hm & 0xffu) << 37);
}

struct ScanSmem {
  float2 col[kBufs][256];   // {a_j, s_j}
  float2 row[kBufs][32];    // {c_i, s_i}
  float4 ctl[kBufs];        // {thr, active, -, -}
};

template <int NC>
__device__ __forceinline__ void scan_task(const DevPtrs& P, const InstDesc& d, int row0, int c0, ScanSmem& sm) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, t = threadIdx.x;
  const int n = d.n, np = d.n_pad, R = P.R, NPs = P.NP, cap = P.cap;
  const int b0 = d.first_search;
  const float* J4 = P.J4 + d.off_mat;
  const float2* as_base = P.as32;
  const float2* cs_base = P.cs32;
  const float4* ctl_base = P.sctl;
  const float qnan = __int_as_float(0x7fc00000);
  const int i0 = row0 + warp * 8;
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
  // stage search s into buffer q: columns (16 bytes = 2 sites per thread), rows (16 threads),
  // {thr, active} (one thread)
  const int col = c0 + 2 * t;
  auto stage = [&](int s, int q) {
    const long long b = b0 + s;
    if (t < 16 * NC) cp_async16(&sm.col[q][2 * t], as_base + b * NPs + min(col, NPs - 2), col < NPs);
    if (t < 16) cp_async16(&sm.row[q][2 * t], cs_base + b * NPs + row0 + 2 * t, true);
    if (t == 16) cp_async16(&sm.ctl[q], ctl_base + b, true);
    cp_async_commit();
  };
  stage(0, 0);
  if (R > 1) stage(1, 1);
  int q = 0;
  for (int s = 0; s < R; ++s) {
    // own copies of search s complete (s+1 may still be in flight); the barrier makes every
    // thread's copies visible and guarantees that all warps have left iteration s-1, whose
    // buffer (s+2) % 3 is restaged right after
    if (s + 1 < R) cp_async_wait<1>();
    else cp_async_wait<0>();
    __syncthreads();
    if (s + 2 < R) stage(s + 2, q == 0 ? 2 : q - 1);
    const float4 ctl = sm.ctl[q];
    if (__any_sync(0xffffffffu, ctl.y != 0.f)) {   // vote result: uniform branch
      const float2* cb = sm.col[q];
      const float2 rv = sm.row[q][warp * 8 + (lane & 7)];
      const unsigned smask = __ballot_sync(0xffffffffu, rv.y < 0.f) & 0xffu;   // bit r: s_i = -1
      float aj[NC], sj[NC];
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        const float2 v = cb[32 * k + lane];
        aj[k] = v.x;
        sj[k] = v.y;
      }
      unsigned hm = 0;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const float c = __shfl_sync(0xffffffffu, rv.x, r);
        float y[NC];
        if ((smask >> r) & 1u) {
#pragma unroll
          for (int k = 0; k < NC; ++k) y[k] = fmaf(-J[r][k], sj[k], aj[k]);
        } else {
#pragma unroll
          for (int k = 0; k < NC; ++k) y[k] = fmaf(J[r][k], sj[k], aj[k]);
        }
        if (rowmin<NC>(y) <= c) hm |= 1u << r;
      }
      const unsigned hit = __ballot_sync(0xffffffffu, hm != 0);
      if (hit) {
        const int b = b0 + s;
        const int leader = __ffs(hit) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(P.surv_cnt + b, __popc(hit));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (hm) {
          const int slot = base + __popc(hit & ((1u << lane) - 1));
          if (slot < cap) P.surv[(long long)b * cap + slot] = make_record(i0, c0 + lane, NC, hm);
        }
      }
    }
    q = (q == kBufs - 1) ? 0 : q + 1;
  }
}

// task.x = instance, task.y = first row of the 32-row block, task.z = first column, task.w = NC
__global__ void __launch_bounds__(128, 4) k_scan_pairs(DevPtrs P, const int4* tasks, int n_tasks) {
  __shared__ __align__(16) ScanSmem sm;
  const int4 w = tasks[blockIdx.x];
  const InstDesc d = P.inst[w.x];
  switch (w.w) {
    case 8: scan_task<8>(P, d, w.y, w.z, sm); break;
    case 4: scan_task<4>(P, d, w.y, w.z, sm); break;
    case 2: scan_task<2>(P, d, w.y, w.z, sm); break;
    default: scan_task<1>(P, d, w.y, w.z, sm); break;
  }
}

cudaError_t launch_scan_pairs(const DevPtrs& P, const int4* tasks, int n_tasks, cudaStream_t s) {
  if (n_tasks <= 0) return cudaSuccess;
  k_scan_pairs<<<n_tasks, 128, 0, s>>>(P, tasks, n_tasks);
  return cudaGetLastError();
}

// Host: cover the pairs (i < j) of an n-spin instance with block tasks. Block a holds rows
// [32a, 32a+32); its columns run from 32a (the 32 x 32 diagonal block is masked inside the
// task) to n, in chunks of 256 columns and then one narrower chunk for the remainder.
void scan_tasks_for(int inst, int n, std::vector<int4>& out) {
  for (int row0 = 0; row0 < n - 1; row0 += 32) {
    int c = row0;
    while (c < n) {
      const int rem = n - c;
      int nc;
      if (rem >= 192) nc = 8;
      else if (rem >= 96) nc = 4;
      else if (rem >= 48) nc = 2;
      else nc = 1;
      out.push_back(make_int4(inst, row0, c, nc));
      c += 32 * nc;
    }
  }
}

}  // namespace qis
