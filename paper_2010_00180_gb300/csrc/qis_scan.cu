// qis_scan.cu -- candidate scan of the split / integer precision modes (FP32 filter).
//
// Pair candidates (i, j), i < j, of one parent: dE_ij = a_i + a_j + 4 s_i s_j J_ij (Sec. III,
// energy change from the couplings of the flipped sites). A pair survives the filter when
// dE~_ij <= thr (per search; k_bound derives thr and the error band it carries).
//
// Work unit = one block task: 32 consecutive rows i (4 warps x 8 rows) and a chunk of 32*NC
// columns j of one instance, for all R searches of that instance. Each lane keeps its 8 x NC
// couplings 4J~_ij in registers and reuses them for every search; lane l owns columns
// c0 + 32k + l. The per-search data -- {a_j, s_j} of the chunk's columns and of the block's
// rows -- is staged into shared memory with cp.async, one search ahead (double buffer).
//
// Per search and row i (warp-uniform), each lane evaluates
//     y_ij = a_j + (s_i s_j) 4J~_ij  = fma(+-4J~_ij, s_j, a_j)
// where the row spin picks the sign of the coupling operand (uniform branch), reduces
// min_j y_ij with three-input minima and tests it against thr - a_i. Pairs that must not be
// evaluated (j <= i, j >= n) hold NaN couplings: the FMA propagates NaN and min ignores it.
// A lane whose rows hit appends one record {rows, its columns, row mask}; the merge expands
// it with the same FP32 test, so the filter decision is identical in both places.
#include "qis_common.cuh"

namespace qis {

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
    const float t0 = min3f(y[0], y[1], y[2]);
    const float t1 = min3f(y[3], y[4], y[5]);
    return min3f(t0, t1, fminf(y[6], y[7]));
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

// Record layout of a scan hit (bit 63 set): bits 0-15 first row of the lane's 8 rows,
// bits 16-31 column of k = 0, bits 32-35 NC, bits 36-43 mask of the rows that hit.
__host__ __device__ inline unsigned long long make_record(int i0, int jb, int nc, unsigned hm) {
  return (1ull << 63) | (unsigned long long)(unsigned)i0 | ((unsigned long long)(unsigned)jb << 16) |
         ((unsigned long long)(unsigned)nc << 32) | ((unsigned long long)(hm & 0xffu) << 36);
}

template <int NC>
__device__ __forceinline__ void scan_task(const DevPtrs& P, const InstDesc& d, int row0, int c0) {
  __shared__ __align__(16) float2 colbuf[2][256];
  __shared__ __align__(16) float2 rowbuf[2][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = d.n, np = d.n_pad;
  const float* J4 = P.J4 + d.off_mat;
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
  // stage search s into buffer s & 1 (columns: 16 bytes = 2 sites per thread; rows: 16 threads)
  auto stage = [&](int s) {
    const int b = d.first_search + s;
    const float2* as = P.as32 + (long long)b * P.NP;
    const int t = threadIdx.x;
    if (t < 16 * NC) {
      const int col = c0 + 2 * t;
      cp_async16(&colbuf[s & 1][2 * t], as + min(col, P.NP - 2), col < P.NP);
    }
    if (t < 16) cp_async16(&rowbuf[s & 1][2 * t], as + row0 + 2 * t, true);
    cp_async_commit();
  };
  stage(0);
  for (int s = 0; s < P.R; ++s) {
    const int b = d.first_search + s;
    if (s + 1 < P.R) {
      stage(s + 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    if (P.active[b]) {
      const float thr = P.thr32[b];
      const float2* cb = colbuf[s & 1];
      const float2* rb = rowbuf[s & 1] + warp * 8;
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
        const float2 ri = rb[r];                 // {a_i, s_i}, same for every lane
        float y[NC];
        if (ri.y < 0.f) {
#pragma unroll
          for (int k = 0; k < NC; ++k) y[k] = fmaf(-J[r][k], sj[k], aj[k]);
        } else {
#pragma unroll
          for (int k = 0; k < NC; ++k) y[k] = fmaf(J[r][k], sj[k], aj[k]);
        }
        if (rowmin<NC>(y) <= thr - ri.x) hm |= 1u << r;
      }
      const unsigned hit = __ballot_sync(0xffffffffu, hm != 0);
      if (hit) {
        int base = 0;
        if (lane == __ffs(hit) - 1) base = atomicAdd(P.surv_cnt + b, __popc(hit));
        base = __shfl_sync(0xffffffffu, base, __ffs(hit) - 1);
        if (hm) {
          const int slot = base + __popc(hit & ((1u << lane) - 1));
          if (slot < P.cap) P.surv[(long long)b * P.cap + slot] = make_record(i0, c0 + lane, NC, hm);
        }
      }
    }
    __syncthreads();   // buffer s & 1 is restaged by iteration s + 1
  }
}

// task.x = instance, task.y = first row of the 32-row block, task.z = first column, task.w = NC
__global__ void __launch_bounds__(128, 4) k_scan_pairs(DevPtrs P, const int4* tasks, int n_tasks) {
  const int4 w = tasks[blockIdx.x];
  const InstDesc d = P.inst[w.x];
  switch (w.w) {
    case 8: scan_task<8>(P, d, w.y, w.z); break;
    case 4: scan_task<4>(P, d, w.y, w.z); break;
    case 2: scan_task<2>(P, d, w.y, w.z); break;
    default: scan_task<1>(P, d, w.y, w.z); break;
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
