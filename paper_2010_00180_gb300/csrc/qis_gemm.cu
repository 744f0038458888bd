// qis_gemm.cu -- exact local fields on the 5th-generation tensor cores (tcgen05 + TMA + TMEM).
//
// The couplings of an instance are held on a fixed-point grid, Jq = J 2^q (int64), and written
// in balanced base-4096 digits, Jq = sum_d 4096^d D_d with D_d in [-2048, 2047]; every digit is
// an exact FP16 integer. With the parent spins S (+-1, FP16) of the R searches of the instance,
//     F_d = D_d S^T            (one FP16 GEMM per digit, FP32 accumulation in TMEM)
// is exact: every product is an integer of magnitude <= 2048 and every partial sum stays below
// 2048 n <= 2^24, so no rounding can occur whatever order the tensor core adds in. The exact
// field of site i for search r is then fq = hq_i + sum_d 4096^d F_d[i][r] (int64) and the
// single-flip energy change a_i = -2 s_i f_i (Sec. III) follows exactly.
//
// Persistent kernel, one CTA per SM, walking 128-row x NT-search tiles of all instances:
//   warp 0 lane 0 : producer: one bulk copy (TMA engine) per digit tile of 128 x 64 and one for
//                   the spin tile NT x 64 per stage -- both operands are stored pre-tiled in the
//                   swizzled shared-memory image (d16_offset, s16_offset), so every copy is
//                   contiguous; one ring of stages runs across tile boundaries
//   warp 1 lane 0 : MMA issuer (tcgen05.mma kind::f16, M=128, N=NT, K=16); tile number lt
//                   accumulates into TMEM buffer lt % 2, so one tile's epilogue overlaps the
//                   next tile's loads and MMAs
//   warps 2-5     : epilogue, each on its TMEM lane quarter: stage the tile's parent spins and
//                   active flags in shared memory, tcgen05.ld the accumulators, exact int64
//                   combination of the digits, a_i = -2 s_i f_i; release the buffer.
// Every wait is bounded (P.wait_ns of %globaltimer, 2 s by default); on timeout the CTA raises
// kStatTimeout, drains what it issued (those waits bounded by a fixed 2 s: the copies and MMAs
// in flight complete), frees its TMEM and returns. P.wait_probe makes the MMA thread first wait
// on a barrier that nothing completes, so that path can be tested without any fault.
#include <cuda_fp16.h>

#include "qis_common.cuh"

namespace qis {

constexpr int kStages = 6;         // most stages of the smem ring
constexpr int kKC = 64;              // K elements per stage (128 bytes of FP16: one swizzle row)
constexpr int kTileBytesA = 128 * kKC * 2;

struct GemmArgs {
  int n_inst, R, NP, Wmax, NT, digits_max, stages, nbuf;
  long long plane;        // halves of one digit plane (every instance's NP x NP tiles)
  long long s16_stride;   // halves of one instance's spin region
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
  return ok != 0;
}
// Bounded wait: false once `limit` ns have passed since t0.
constexpr uint64_t kDrainNs = 2000000000ull;   // bound of the waits for work already issued (2 s)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t t0, uint64_t limit) {
  while (!mbar_try(bar, parity)) {
    if (gtimer() - t0 > limit) return false;
  }
  return true;
}
// 1-D bulk copy global -> shared (TMA engine); completion counted in bytes on the mbarrier
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
// K-major operand tile, 128-byte rows, 128B swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);          // start address
  d |= (uint64_t)(16u >> 4) << 16;                    // leading byte offset (unused for SW128 K-major)
  d |= (uint64_t)(1024u >> 4) << 32;                  // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                             // fixed 0b001
  d |= (uint64_t)2 << 61;                             // SWIZZLE_128B
  return d;
}
// kind::f16 instruction descriptor: D = F32, A = B = F16, K-major both, N, M = 128.
__device__ __forceinline__ uint32_t idesc_f16(int N) {
  return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(tmem_d), "l"(da), "l"(db), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
// Barrier of the four epilogue warps that also ORs a flag over them: every epilogue thread gets
// the same answer, so they all leave their loop at the same tile (no one is left at a barrier).
__device__ __forceinline__ bool epi_vote(bool flag) {
  uint32_t any;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, 128, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(any) : "r"((uint32_t)flag) : "memory");
  return any != 0;
}

// Persistent: one CTA per SM walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ...; tile t is
// (instance t / tpi, 128-row block, NT-search block), tpi = (NP / 128) * ceil(R / NT); row blocks
// at or past an instance's n_pad are skipped by every role alike.
__global__ void __launch_bounds__(192, 1) k_fields_tc(const __half* __restrict__ D16, const __half* __restrict__ S16,
                                                      DevPtrs P, GemmArgs G) {
  const int NT = G.NT, S = G.stages, Dm = G.digits_max, nbuf = G.nbuf;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int bytesB = NT * kKC * 2;
  const int stage_bytes = Dm * kTileBytesA + bytesB;   // same layout for every instance
  const int n_mt = G.NP / 128, n_nt = (G.R + NT - 1) / NT, tpi = n_mt * n_nt;
  // with fields by update, only the tiles holding a search that needs full fields (every role
  // reads the same flags, written by the previous kernel)
  auto skip = [&](int tile) { return P.inc_on && !P.full_tile[(tile / tpi) * n_nt + tile % n_nt]; };
  const int n_tiles = G.n_inst * tpi;

  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], tfull[2], tempty[2], done, never;
  __shared__ uint32_t tmem_base;
  __shared__ int s_err;
  __shared__ uint64_t s_pw[256][2];   // parent spin words of the tile's rows, per search of the tile
  __shared__ int s_act[256];          // active flag per search of the tile
  __shared__ int s_it[256];           // its iteration (the aq ring slot)
  int ncols = 32;
  while (ncols < nbuf * Dm * NT) ncols <<= 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4);   // one arrival per epilogue warp
    }
    mbar_init(&done, 1);
    mbar_init(&never, 1);   // no thread ever arrives here (the timeout probe)
    s_err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint64_t t0 = gtimer();

  if (threadIdx.x == 0) {
    // ---------------- TMA producer: the k-blocks of every tile, one stage ring across tiles
    int it = 0;
    for (int tile = blockIdx.x; tile < n_tiles && !*(volatile int*)&s_err; tile += gridDim.x) {
      const int inst = tile / tpi, m0 = ((tile % tpi) / n_nt) * 128, n0 = (tile % n_nt) * NT;
      const InstDesc d = P.inst[inst];
      if (m0 >= d.n_pad || skip(tile)) continue;
      const int kc_total = d.n_pad / kKC;
      for (int kc = 0; kc < kc_total; ++kc, ++it) {
        const int s = it % S;
        if (it >= S && !mbar_wait(&empty[s], ((it / S) + 1) & 1, t0, P.wait_ns)) {
          atomicOr(&s_err, 1);
          break;
        }
        if (*(volatile int*)&s_err) break;
        unsigned char* st = smem + s * stage_bytes;
        mbar_expect_tx(&full[s], (uint32_t)(d.digits * kTileBytesA + bytesB));
        // pre-tiled operands (d16_offset / s16_offset): one contiguous bulk copy per tile
        const long long ta = ((long long)(m0 >> 7) * (G.NP >> 6) + kc) * 8192;
        for (int dg = 0; dg < d.digits; ++dg)
          bulk_g2s(st + dg * kTileBytesA, D16 + dg * G.plane + (long long)inst * G.NP * G.NP + ta,
                   (uint32_t)kTileBytesA, &full[s]);
        const long long tb = ((long long)(n0 / NT) * (G.NP >> 6) + kc) * ((long long)NT * 64);
        bulk_g2s(st + Dm * kTileBytesA, S16 + (long long)inst * G.s16_stride + tb, (uint32_t)bytesB, &full[s]);
      }
    }
    // drain: after an error the last (at most S) issued stages may still be in flight; each
    // stage's full barrier is in the phase armed last, so the parity waits are exact
    if (*(volatile int*)&s_err) {
      for (int k = max(0, it - S); k < it; ++k) mbar_wait(&full[k % S], (k / S) & 1, gtimer(), kDrainNs);
    }
  } else if (threadIdx.x == 32) {
    // ---------------- MMA issuer: tile lt accumulates into TMEM buffer lt % nbuf
    const uint32_t idesc = idesc_f16(NT);
    int it = 0, lt = 0;
    if (P.wait_probe && !mbar_wait(&never, 0, t0, P.wait_ns)) atomicOr(&s_err, 8);   // always runs out
    for (int tile = blockIdx.x; tile < n_tiles && !*(volatile int*)&s_err; tile += gridDim.x) {
      const int inst = tile / tpi, m0 = ((tile % tpi) / n_nt) * 128;
      const InstDesc d = P.inst[inst];
      if (m0 >= d.n_pad || skip(tile)) continue;
      const int buf = lt % nbuf, use = lt / nbuf;
      if (use > 0 && !mbar_wait(&tempty[buf], (use - 1) & 1, t0, P.wait_ns)) {
        atomicOr(&s_err, 2);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t acc = tmem + (uint32_t)(buf * Dm * NT);
      const int kc_total = d.n_pad / kKC;
      bool ok = true;
      for (int kc = 0; kc < kc_total; ++kc, ++it) {
        const int s = it % S;
        if (!mbar_wait(&full[s], (it / S) & 1, t0, P.wait_ns)) {
          atomicOr(&s_err, 2);
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        unsigned char* st = smem + s * stage_bytes;
        const uint32_t b_addr = smem_u32(st + Dm * kTileBytesA);
        for (int dg = 0; dg < d.digits; ++dg) {
          const uint32_t a_addr = smem_u32(st + dg * kTileBytesA);
#pragma unroll
          for (int k4 = 0; k4 < kKC / 16; ++k4)
            mma_f16(acc + dg * NT, sdesc(a_addr + k4 * 32), sdesc(b_addr + k4 * 32), idesc, (kc | k4) != 0);
        }
        mma_commit(&empty[s]);   // stage free once these MMAs have read it
      }
      if (!ok) break;
      mma_commit(&tfull[buf]);   // the tile's accumulators are complete
      ++lt;
    }
    mma_commit(&done);           // every MMA issued so far completes -> done
    mbar_wait(&done, 0, gtimer(), kDrainNs);
  } else if (warp >= 2) {
    // ---------------- epilogue warps 2-5: TMEM lane quarter (warp % 4), exact int64 fields
    const int quarter = warp & 3, etid = threadIdx.x - 64;
    int lt = 0;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
      const int inst = tile / tpi, m0 = ((tile % tpi) / n_nt) * 128, n0 = (tile % n_nt) * NT;
      const InstDesc d = P.inst[inst];
      if (m0 >= d.n_pad || skip(tile)) continue;
      const int buf = lt % nbuf, use = lt / nbuf;
      // the tile's per-search inputs, staged while its accumulators are being computed
      epi_bar();   // every epilogue warp is done with the previous tile's copy
      const int w0 = m0 >> 6;
      for (int t = etid; t < NT; t += 128) {
        const int r = n0 + t;
        const long long b = d.first_search + r;
        const bool valid = r < G.R;
        s_act[t] = valid ? P.active[b] : 0;
        s_it[t] = valid ? P.iter_t[b] : 0;
        s_pw[t][0] = valid ? P.par_bits[b * G.Wmax + w0] : 0ull;
        s_pw[t][1] = (valid && w0 + 1 < G.Wmax) ? P.par_bits[b * G.Wmax + w0 + 1] : 0ull;
      }
      const bool ok = mbar_wait(&tfull[buf], use & 1, t0, P.wait_ns);
      if (epi_vote(!ok || *(volatile int*)&s_err != 0)) {   // also orders the staging above
        if (!ok) atomicOr(&s_err, 4);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int row = quarter * 32 + lane;
      const int i = m0 + row;
      const float scale_q = (float)d.inv_scale;   // 2^-q, exact in FP32 (q <= 64)
      const long long hq = (i < d.n) ? P.hq[d.off_vec + i] : 0;
      for (int c0 = 0; c0 < NT; c0 += 16) {
        long long acc[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) acc[u] = hq;
        long long wdig = 1;
        for (int dg = 0; dg < d.digits; ++dg) {
          uint32_t v[16];
          const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * Dm * NT + dg * NT + c0);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
              : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int u = 0; u < 16; ++u) acc[u] += wdig * (long long)__float2int_rn(__uint_as_float(v[u]));
          wdig <<= d.dbits;
        }
        if (i < d.n_pad) {
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const int t = c0 + u;
            if (n0 + t >= G.R || !s_act[t]) continue;
            const long long b = d.first_search + n0 + t;
            long long aq = 0;
            float2 as = make_float2(0.f, 0.f);
            if (i < d.n) {
              const int sg = (int)((s_pw[t][row >> 6] >> (row & 63)) & 1ull);   // sigma_i of the parent
              aq = sg ? 2 * acc[u] : -2 * acc[u];
              // fl32(aq 2^-q) = fl32(aq) 2^-q: scaling by a power of two commutes with rounding
              as = make_float2(__ll2float_rn(aq) * scale_q, sg ? -1.f : 1.f);
            }
            aq_of(P, b, s_it[t])[i] = aq;
            P.as32[b * P.NP + i] = as;
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[buf])) : "memory");
      ++lt;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (s_err && threadIdx.x == 0) atomicOr(P.status, kStatTimeout);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// ---------------------------------------------------------------- host side
// Searches per tile: a multiple of 16 with two accumulator sets in TMEM (2 * digits * nt <= 512
// columns) when possible, else one; among those the one that pads R the least, then the widest.
int gemm_tile_n(int R, int digits) {
  int cap = 512 / (2 * digits) / 16 * 16;
  if (cap < 16) cap = 512 / digits / 16 * 16;
  if (cap > 256) cap = 256;
  int best = 16, best_pad = 1 << 30;
  for (int nt = 16; nt <= cap; nt += 16) {
    const int pad = (R + nt - 1) / nt * nt;
    if (pad < best_pad || (pad == best_pad && nt > best)) {
      best = nt;
      best_pad = pad;
    }
  }
  return best;
}

// As many stages as fit in ~200 KB of shared memory (one CTA per SM), at most kStages.
int gemm_stages(int digits, int nt) {
  const size_t per = (size_t)digits * kTileBytesA + (size_t)nt * kKC * 2;
  int st = (int)((200 * 1024) / per);
  if (st > kStages) st = kStages;
  if (st < 2) st = 2;
  return st;
}

size_t gemm_smem(int digits, int nt) {
  return (size_t)gemm_stages(digits, nt) * (digits * kTileBytesA + nt * kKC * 2) + 1024;
}

// nt: searches per tile (multiple of 16, digits_max * nt <= 512), or 0 for gemm_tile_n's choice.
cudaError_t launch_fields_tc(const DevPtrs& P, const void* D16, const void* S16, int max_inst, int digits_max,
                             int nt, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  GemmArgs G;
  G.n_inst = P.n_inst;
  G.R = P.R;
  G.NP = P.NP;
  G.Wmax = P.Wmax;
  G.digits_max = digits_max;
  G.plane = (long long)max_inst * P.NP * P.NP;
  G.s16_stride = P.s16_stride;
  G.NT = nt > 0 ? nt : gemm_tile_n(P.R, digits_max);
  G.stages = gemm_stages(digits_max, G.NT);
  G.nbuf = (2 * digits_max * G.NT <= 512) ? 2 : 1;   // double-buffered accumulators if TMEM holds two
  const size_t sm = gemm_smem(digits_max, G.NT);
  static size_t attr = 0;
  if (attr < sm) {
    e = cudaFuncSetAttribute(k_fields_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr = sm;
  }
  static int n_sm = 0;
  if (n_sm == 0) {
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
  }
  const int tiles = P.n_inst * (P.NP / 128) * ((P.R + G.NT - 1) / G.NT);
  const int grid = tiles < n_sm ? tiles : n_sm;
  if (grid <= 0) return cudaSuccess;
  k_fields_tc<<<grid, 192, sm, s>>>(static_cast<const __half*>(D16), static_cast<const __half*>(S16), P, G);
  return cudaGetLastError();
}

}  // namespace qis
