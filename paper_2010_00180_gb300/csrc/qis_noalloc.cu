// qis_noalloc.cu -- candidate selection of one parent state without any device allocation.
//
// Some callers cannot call cudaMalloc at the moment they need this work done: code that runs
// while a CUDA stream is being captured into a graph (an allocation there breaks the capture),
// real-time loops that must never block in the driver's allocator, and plugins that live in a
// host process whose device memory is owned by another framework's pool. For them this file
// keeps the one scratch area it needs in a file-scope __device__ array, sized at build time;
// the caller passes only its own input and output buffers.
//
// What it computes (FP64, the same arithmetic as the library's QIS_FP64 mode): for a parent
// state psi of an n-spin instance (J, h), every single flip i and pair flip i < j, with
// E' = E(psi) + dE, and returns the k candidates of lowest (E', c), c the candidate index
// (c = i for singles, n + rank(i, j) for pairs). This is the candidate side of one iteration
// of the QI search before duplicates against a kept list are removed.
//
// The scratch array is shared by every call on a device and keeps the last call's contents;
// every element a call reads is written earlier in that same call, so nothing needs clearing.
// Calls whose kernels overlap on the GPU (different streams, no ordering) race on the array.
#include <mutex>
#include <string>

#include "qis_common.cuh"

namespace qis {

constexpr int kNaMaxN = 512;       // largest n accepted
constexpr int kNaMaxK = 128;       // largest k accepted
constexpr int kNaBlocks = 64;      // candidate blocks (each keeps its own k lowest)
constexpr int kNaChunk = 4096;     // >= ceil(n(n+1)/2 / kNaBlocks) for n <= kNaMaxN, power of two

struct NoAllocScratch {
  double a[kNaMaxN];                         // a_i = -2 s_i f_i of the parent
  double Ep;                                 // E(psi)
  double E[kNaBlocks][kNaMaxK];              // per-block k lowest energies
  uint32_t c[kNaBlocks][kNaMaxK];            // and their candidate indices
};

// ~100 KB; every GPU that loads the library holds it until the process exits
static __device__ __align__(256) NoAllocScratch g_na_scratch;

// f_i = (sum_{j != i} s_j J_ij, j ascending) + h_i, a_i = -2 s_i f_i; E(psi) = pair sum
// (i-major, j ascending) + field sum, all in FP64 with unfused additions.
__global__ void __launch_bounds__(256) k_na_fields(int n, const double* J, const double* h, const uint64_t* bits,
                                                   NoAllocScratch* S) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      const double v = J[(long long)i * n + j];
      acc = __dadd_rn(acc, sigma_of(bits, j) ? -v : v);
    }
    const double f = __dadd_rn(acc, h[i]);
    S->a[i] = sigma_of(bits, i) ? 2.0 * f : -2.0 * f;
  }
  if (threadIdx.x == 0) {
    double Pp = 0.0, F = 0.0;
    for (int i = 0; i < n; ++i) {
      const double si = sigma_of(bits, i) ? -1.0 : 1.0;
      for (int j = i + 1; j < n; ++j) Pp = __dadd_rn(Pp, J[(long long)i * n + j] * si * (sigma_of(bits, j) ? -1.0 : 1.0));
    }
    for (int i = 0; i < n; ++i) F = __dadd_rn(F, h[i] * (sigma_of(bits, i) ? -1.0 : 1.0));
    S->Ep = __dadd_rn(Pp, F);
  }
}

__device__ void na_sort(unsigned long long* key, uint32_t* val, int n2) {
  for (int k = 2; k <= n2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < n2; t += blockDim.x) {
        const int u = t ^ j;
        if (u > t) {
          const unsigned long long a = key[t], c = key[u];
          const uint32_t va = val[t], vc = val[u];
          const bool gt = (a > c) || (a == c && va > vc);
          if (gt == ((t & k) == 0)) {
            key[t] = c; key[u] = a;
            val[t] = vc; val[u] = va;
          }
        }
      }
      __syncthreads();
    }
  }
}

// Block b handles the candidate indices [b*chunk, (b+1)*chunk) and keeps its k lowest (E', c).
__global__ void __launch_bounds__(256) k_na_candidates(int n, const double* J, const uint64_t* bits, int k,
                                                       NoAllocScratch* S) {
  extern __shared__ __align__(16) unsigned char na_smem[];
  unsigned long long* key = reinterpret_cast<unsigned long long*>(na_smem);   // [kNaChunk]
  uint32_t* val = reinterpret_cast<uint32_t*>(key + kNaChunk);                // [kNaChunk]
  const long long C = (long long)n * (n + 1) / 2;
  const int chunk = (int)((C + kNaBlocks - 1) / kNaBlocks);
  const long long lo = (long long)blockIdx.x * chunk;
  const double Ep = S->Ep;
  for (int t = threadIdx.x; t < kNaChunk; t += blockDim.x) {
    unsigned long long kk = ~0ull;
    uint32_t c = 0xffffffffu;
    const long long cc = lo + t;
    if (t < chunk && cc < C) {
      c = (uint32_t)cc;
      int i, j;
      decode_candidate(n, c, i, j);
      double de = S->a[i];
      if (j >= 0) de = dE64(S->a[i], S->a[j], J[(long long)i * n + j], sigma_of(bits, i) ^ sigma_of(bits, j));
      kk = dkey(__dadd_rn(Ep, de));
    }
    key[t] = kk;
    val[t] = c;
  }
  __syncthreads();
  na_sort(key, val, kNaChunk);
  for (int t = threadIdx.x; t < k; t += blockDim.x) {
    S->E[blockIdx.x][t] = (key[t] == ~0ull) ? INFINITY : dkey_inv(key[t]);
    S->c[blockIdx.x][t] = val[t];
  }
}

// Merge of the per-block lists: the k lowest (E', c) overall.
__global__ void __launch_bounds__(256) k_na_final(int k, NoAllocScratch* S, double* E_out, uint32_t* c_out,
                                                  double* Ep_out) {
  extern __shared__ __align__(16) unsigned char na_smem[];
  const int m = kNaBlocks * k, m2 = next_pow2(m);
  unsigned long long* key = reinterpret_cast<unsigned long long*>(na_smem);   // [m2]
  uint32_t* val = reinterpret_cast<uint32_t*>(key + m2);                      // [m2]
  for (int t = threadIdx.x; t < m2; t += blockDim.x) {
    unsigned long long kk = ~0ull;
    uint32_t c = 0xffffffffu;
    if (t < m) {
      const int blk = t / k, r = t % k;
      c = S->c[blk][r];
      if (c != 0xffffffffu) kk = dkey(S->E[blk][r]);
    }
    key[t] = kk;
    val[t] = c;
  }
  __syncthreads();
  na_sort(key, val, m2);
  for (int t = threadIdx.x; t < k; t += blockDim.x) {
    E_out[t] = (key[t] == ~0ull) ? INFINITY : dkey_inv(key[t]);
    c_out[t] = val[t];
  }
  if (threadIdx.x == 0 && Ep_out) *Ep_out = S->Ep;
}

namespace {
std::mutex g_na_mu;
NoAllocScratch* g_na_ptr[64] = {nullptr};   // device address of the scratch array, per device
bool g_na_attr[64] = {false};
}  // namespace

}  // namespace qis

using namespace qis;

extern "C" int qis_select_candidates_noalloc(int n, const double* J, const double* h, const uint64_t* bits, int k,
                                             double* E_out, uint32_t* c_out, double* Ep_out, void* stream) {
  if (n < 2 || n > kNaMaxN) {
    set_global_error("qis_select_candidates_noalloc: n must be in [2, 512] (static scratch size)");
    return QIS_ERR_INVALID_ARG;
  }
  if (k < 1 || k > kNaMaxK || (long long)k > (long long)n * (n + 1) / 2) {
    set_global_error("qis_select_candidates_noalloc: k must be in [1, min(128, n(n+1)/2)] (static scratch size)");
    return QIS_ERR_INVALID_ARG;
  }
  if (!J || !h || !bits || !E_out || !c_out) {
    set_global_error("qis_select_candidates_noalloc: NULL buffer");
    return QIS_ERR_INVALID_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    set_global_error("qis_select_candidates_noalloc: no current CUDA device");
    return QIS_ERR_CUDA;
  }
  NoAllocScratch* S = nullptr;
  {
    // set-up once per device, with that device current: the host-side name of the array is a
    // stand-in, the kernels need its device address
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
      if (e != cudaSuccess || !p) {
        set_global_error((std::string("qis_select_candidates_noalloc: cudaGetSymbolAddress of the scratch array: ") +
                          cudaGetErrorString(e)).c_str());
        return QIS_ERR_CUDA;
      }
      g_na_ptr[dev] = static_cast<NoAllocScratch*>(p);
    }
    if (!g_na_attr[dev]) {
      const int sm_c = kNaChunk * 12, sm_f = next_pow2(kNaBlocks * kNaMaxK) * 12;
      cudaError_t e = cudaFuncSetAttribute(k_na_candidates, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_c);
      if (e == cudaSuccess) e = cudaFuncSetAttribute(k_na_final, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_f);
      if (e != cudaSuccess) {
        set_global_error((std::string("qis_select_candidates_noalloc: shared-memory attribute: ") +
                          cudaGetErrorString(e)).c_str());
        return QIS_ERR_CUDA;
      }
      g_na_attr[dev] = true;
    }
    S = g_na_ptr[dev];
  }
  // Each launch's own status: cudaLaunchKernel returns the error of that launch (it does not
  // consume an error the caller's earlier work left in the runtime's last-error state).
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const auto launched = [](cudaError_t e, const char* kernel) {
    if (e == cudaSuccess) return QIS_OK;
    set_global_error((std::string("qis_select_candidates_noalloc: launch of ") + kernel + ": " +
                      cudaGetErrorString(e)).c_str());
    return QIS_ERR_CUDA;
  };
  {
    void* args[] = {&n, &J, &h, &bits, &S};
    const int rc = launched(cudaLaunchKernel((const void*)k_na_fields, dim3(1), dim3(256), args, 0, s), "k_na_fields");
    if (rc) return rc;
  }
  {
    void* args[] = {&n, &J, &bits, &k, &S};
    const int rc = launched(cudaLaunchKernel((const void*)k_na_candidates, dim3(kNaBlocks), dim3(256), args,
                                             (size_t)kNaChunk * 12, s), "k_na_candidates");
    if (rc) return rc;
  }
  {
    void* args[] = {&k, &S, &E_out, &c_out, &Ep_out};
    return launched(cudaLaunchKernel((const void*)k_na_final, dim3(1), dim3(256), args,
                                     (size_t)next_pow2(kNaBlocks * k) * 12, s), "k_na_final");
  }
}
