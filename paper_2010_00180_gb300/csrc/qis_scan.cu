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
// A warp with a hit recomputes, on that rare path, each lane's exact (row, column) hits with
// the same FP32 expression and appends one survivor entry per passing pair.
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

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  const int sz = valid ? 16 : 0;   // 0 bytes read -> 16 zero bytes written
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(sz) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

struct ScanSmem {
  float2 col[kBufs][256];   // {a_j, s_j}
  float2 row[kBufs][32];    // {c_i, s_i}
  float4 ctl[kBufs];        // {thr, active, RD(min_j a_j - j4max), -}
};

template <int NC>
__device__ __forceinline__ void scan_task(const DevPtrs& P, const InstDesc& d, int row0, int c0, int g, int RG,
                                          ScanSmem& sm) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, t = threadIdx.x;
  const int n = d.n, np = d.n_pad, NPs = P.NP, cap = P.cap;
  const int b0 = d.first_search + g * RG;        // searches [g RG, g RG + R) of the instance
  const int R = min(RG, P.R - g * RG);
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
    // rows that can hit: y_ij >= RD(min_j a_j - j4max) = ctl.z for every column (rounding is
    // monotone), so a row with c_i < ctl.z has no pair below its bound; skipped rows cost a vote
    const float2 rv = sm.row[q][warp * 8 + (lane & 7)];
    const unsigned live = __ballot_sync(0xffffffffu, ctl.y != 0.f && rv.x >= ctl.z) & 0xffu;
    if (live) {   // vote result: uniform branch
      const float2* cb = sm.col[q];
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
        if (!((live >> r) & 1u)) continue;   // uniform
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
        // rare path: the exact (row, column) hits of this lane, recomputed with the same FP32
        // expression from the couplings still in registers, one survivor entry per pair
        unsigned long long cm = 0;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const float c = __shfl_sync(0xffffffffu, rv.x, r);
          if ((hm >> r) & 1u) {
            const bool neg = (smask >> r) & 1u;
#pragma unroll
            for (int k = 0; k < NC; ++k) {
              const float y = neg ? fmaf(-J[r][k], sj[k], aj[k]) : fmaf(J[r][k], sj[k], aj[k]);
              if (y <= c) cm |= 1ull << (r * NC + k);
            }
          }
        }
        const int mine = __popcll(cm);
        int incl = mine;   // inclusive warp prefix of the per-lane hit counts
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        int base = 0;
        if (lane == 31) base = atomicAdd(P.surv_cnt + b0 + s, incl);
        base = __shfl_sync(0xffffffffu, base, 31);
        int slot = base + incl - mine;
        while (cm) {
          const int bit = __ffsll((long long)cm) - 1;
          cm &= cm - 1;
          const int i = i0 + bit / NC, j = c0 + 32 * (bit % NC) + lane;
          if (slot < cap) P.surv[(long long)(b0 + s) * cap + slot] = surv_entry(pair_index(n, i, j), i, j);
          ++slot;
        }
      }
    }
    q = (q == kBufs - 1) ? 0 : q + 1;
  }
}

// task.x = instance, task.y = first row of the 32-row block, task.z = first column,
// task.w = NC | (search group << 8); a group is RG consecutive searches of the instance
__global__ void __launch_bounds__(128, 4) k_scan_pairs(DevPtrs P, const int4* tasks, int n_tasks, int RG) {
  __shared__ __align__(16) ScanSmem sm;
  const int4 w = tasks[blockIdx.x];
  const InstDesc d = P.inst[w.x];
  const int g = w.w >> 8;
  switch (w.w & 0xff) {
    case 8: scan_task<8>(P, d, w.y, w.z, g, RG, sm); break;
    case 7: scan_task<7>(P, d, w.y, w.z, g, RG, sm); break;
    case 6: scan_task<6>(P, d, w.y, w.z, g, RG, sm); break;
    case 5: scan_task<5>(P, d, w.y, w.z, g, RG, sm); break;
    case 4: scan_task<4>(P, d, w.y, w.z, g, RG, sm); break;
    case 3: scan_task<3>(P, d, w.y, w.z, g, RG, sm); break;
    case 2: scan_task<2>(P, d, w.y, w.z, g, RG, sm); break;
    default: scan_task<1>(P, d, w.y, w.z, g, RG, sm); break;
  }
}

cudaError_t launch_scan_pairs(const DevPtrs& P, const int4* tasks, int n_tasks, int RG, cudaStream_t s) {
  if (n_tasks <= 0) return cudaSuccess;
  k_scan_pairs<<<n_tasks, 128, 0, s>>>(P, tasks, n_tasks, RG);
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
