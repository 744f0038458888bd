// qis_mlp.cu -- learned warm start: a per-site MLP that proposes initial states.
//
// The QI search starts every search from a random state (rand_between of Alg. 4). Here a
// small network maps features of each site (h_i and statistics of row i of J) to a logit
// z_i of P(s_i = +1); the R initial states of an instance are its argmax (search 0) and
// Bernoulli draws from sigmoid(z) (searches 1..R-1). The network is trained on the GPU by
// the kernels below on states the search itself found; random initial states remain the
// default and the reference for comparison.
//
// Network: F = 8 features -> H -> H -> H -> 1, ReLU, BF16 weights (rounded from an FP32
// master copy after every update), FP32 activations and accumulation, BCE loss, Adam.
// Features (FP64, then FP32): h_i, sum_j J_ij / sqrt n, sum_j |J_ij| / n,
// sqrt(sum_j J_ij^2 / n), max_{j!=i} J_ij, min_{j!=i} J_ij, sum_j J_ij h_j / sqrt n,
// sum_j J_ij sign(h_j) / sqrt n.
#include <cuda_bf16.h>
#include <math.h>

#include <string>
#include <vector>

#include "qis_common.cuh"

namespace qis {

constexpr int kF = 8;   // features per site

// ---------------------------------------------------------------- features
// J row i at J + i * stride (n valid entries), h[0..n).
__global__ void k_mlp_features(const double* J, long long stride, const double* h, int n, float* X) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* row = J + (long long)i * stride;
  double s = 0, a = 0, q = 0, mx = -INFINITY, mn = INFINITY, jh = 0, js = 0;
  for (int j = 0; j < n; ++j) {
    const double v = row[j];
    s += v;
    a += fabs(v);
    q += v * v;
    jh += v * h[j];
    js += v * (double)((h[j] > 0) - (h[j] < 0));
    if (j != i) {
      mx = fmax(mx, v);
      mn = fmin(mn, v);
    }
  }
  const double rn = sqrt((double)n);
  float* x = X + (long long)i * kF;
  x[0] = (float)h[i];
  x[1] = (float)(s / rn);
  x[2] = (float)(a / n);
  x[3] = (float)sqrt(q / n);
  x[4] = (float)mx;
  x[5] = (float)mn;
  x[6] = (float)(jh / rn);
  x[7] = (float)(js / rn);
}

__global__ void k_mlp_labels(const uint64_t* bits, int n, float* y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = ((bits[i >> 6] >> (i & 63)) & 1ull) ? 0.f : 1.f;   // y = 1 <=> s_i = +1
}

// ---------------------------------------------------------------- GEMM (SIMT, FP32 accumulate)
// C[M x N] (+)= op(A)[M x K] op(B)[K x N]; A stored [M x K] (TA: [K x M]), B stored [K x N]
// (TB: [N x K]); row-major. Optional epilogue: C = relu(C + bias). gridDim.z splits K and
// accumulates with atomics (C must be zero then).
template <bool TA, bool TB, typename TBt, bool BIAS_RELU>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const float* A, const TBt* B, float* C,
                                              const float* bias) {
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64 + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int kchunk = (K + gridDim.z - 1) / gridDim.z;
  const int k_lo = blockIdx.z * kchunk, k_hi = min(K, k_lo + kchunk);
  float acc[4][4] = {};
  for (int k0 = k_lo; k0 < k_hi; k0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      const int kk = e / 64, mm = e % 64;       // As[kk][mm] = op(A)[m0+mm][k0+kk]
      const int m = m0 + mm, k = k0 + kk;
      float v = 0.f;
      if (m < M && k < k_hi) v = TA ? A[(long long)k * M + m] : A[(long long)m * K + k];
      As[kk][mm] = v;
      const int nn = e % 64, n = n0 + nn;       // Bs[kk][nn] = op(B)[k0+kk][n0+nn]
      float w = 0.f;
      if (n < N && k < k_hi) {
        if constexpr (TB) w = (float)B[(long long)n * K + k];
        else w = (float)B[(long long)k * N + n];
      }
      Bs[kk][nn] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[kk][ty * 4 + u];
        b[u] = Bs[kk][tx * 4 + u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int m = m0 + ty * 4 + u;
    if (m >= M) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int n = n0 + tx * 4 + v;
      if (n >= N) continue;
      if constexpr (BIAS_RELU) {
        C[(long long)m * N + n] = fmaxf(acc[u][v] + bias[n], 0.f);
      } else if (gridDim.z > 1) {
        atomicAdd(&C[(long long)m * N + n], acc[u][v]);
      } else {
        C[(long long)m * N + n] = acc[u][v];
      }
    }
  }
}

// z = h3 w4 + b4 (one output), loss and dz = (sigmoid(z) - y) / M
__global__ void k_mlp_head(int M, int H, const float* h3, const __nv_bfloat16* w4, const float* b4, const float* y,
                           float* z, float* dz, double* loss, float inv_m) {
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (r >= M) return;
  float s = 0.f;
  for (int k = lane; k < H; k += 32) s = fmaf(h3[(long long)r * H + k], __bfloat162float(w4[k]), s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    const float zz = s + b4[0];
    z[r] = zz;
    if (y) {
      const float yy = y[r];
      const float sp = fmaxf(zz, 0.f) + log1pf(expf(-fabsf(zz)));   // softplus
      atomicAdd(loss, (double)(sp - yy * zz) * inv_m);
      dz[r] = (1.f / (1.f + expf(-zz)) - yy) * inv_m;
    }
  }
}

// da3 = outer(dz, w4) * (h3 > 0)
__global__ void k_mlp_head_back(int M, int H, const float* dz, const __nv_bfloat16* w4, const float* h3, float* da) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)M * H) return;
  const int r = (int)(e / H), k = (int)(e % H);
  da[e] = h3[e] > 0.f ? dz[r] * __bfloat162float(w4[k]) : 0.f;
}

__global__ void k_relu_mask(long long count, const float* h, float* d) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count && !(h[e] > 0.f)) d[e] = 0.f;
}

// column sums of d [M x N] into g (atomic)
__global__ void k_colsum(int M, int N, const float* d, float* g) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int rows = (M + gridDim.y - 1) / gridDim.y, r0 = blockIdx.y * rows, r1 = min(M, r0 + rows);
  float s = 0.f;
  for (int r = r0; r < r1; ++r) s += d[(long long)r * N + n];
  atomicAdd(&g[n], s);
}

// dw4 = h3^T dz
__global__ void k_head_wgrad(int M, int H, const float* h3, const float* dz, float* g) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= H) return;
  const int rows = (M + gridDim.y - 1) / gridDim.y, r0 = blockIdx.y * rows, r1 = min(M, r0 + rows);
  float s = 0.f;
  for (int r = r0; r < r1; ++r) s = fmaf(h3[(long long)r * H + k], dz[r], s);
  atomicAdd(&g[k], s);
}

__global__ void k_adam(int count, float* p, const float* g, float* m, float* v, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  const float gg = g[e];
  const float mm = b1 * m[e] + (1.f - b1) * gg;
  const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
  m[e] = mm;
  v[e] = vv;
  p[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

__global__ void k_to_bf16(int count, const float* p, __nv_bfloat16* q) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) q[e] = __float2bfloat16_rn(p[e]);
}

// Initial states from logits: search 0 takes s_i = sign(z_i) (s_i = +1 when z_i >= 0), search
// r >= 1 draws s_i = +1 with probability sigmoid(z_i) using value (r n + i) of the SplitMix64
// stream keyed by `key` (the top 53 bits as a uniform in [0, 1)).
__global__ void k_mlp_sample(const float* z, int n, int R, uint64_t key, uint64_t* bits, int Wstride) {
  const int r = blockIdx.y;
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  const int W = (n + 63) >> 6;
  if (w >= W || r >= R) return;
  uint64_t word = 0;
  for (int b = 0; b < 64; ++b) {
    const int i = w * 64 + b;
    if (i >= n) break;
    int sigma;
    if (r == 0) {
      sigma = z[i] < 0.f;
    } else {
      const double u = (double)(splitmix64(key, (uint64_t)r * n + i) >> 11) * 0x1.0p-53;
      const double p = 1.0 / (1.0 + exp(-(double)z[i]));
      sigma = !(u < p);
    }
    word |= (uint64_t)sigma << b;
  }
  bits[(long long)r * Wstride + w] = word;
}

}  // namespace qis

using namespace qis;

struct qis_mlp {
  qis_mlp_config cfg{};
  int H = 256, F = kF, cap = 0, batch = 0, max_n = 0;
  int n_params = 0;
  cudaStream_t stream = nullptr;
  std::vector<void*> allocs;
  float* P = nullptr;          // master parameters, flattened W1 b1 W2 b2 W3 b3 w4 b4
  float* G = nullptr;          // gradients
  float* Mm = nullptr;         // Adam first moment
  float* Vv = nullptr;         // Adam second moment
  __nv_bfloat16* Pb = nullptr; // BF16 copy of all parameters (biases read from P)
  float* X = nullptr;          // training features [cap x F]
  float* Y = nullptr;          // labels [cap]
  int n_examples = 0;          // rows of X / Y in use
  float *h1 = nullptr, *h2 = nullptr, *h3 = nullptr, *d1 = nullptr, *d2 = nullptr, *zb = nullptr, *dzb = nullptr;
  double* loss = nullptr;
  double* Jst = nullptr;       // staging of one instance's couplings [max_n^2]
  double* hst = nullptr;
  uint64_t* bst = nullptr;
  float* Xq = nullptr;         // query features [max_n x F]
  int adam_t = 0;
  std::string err = "no error";
  // offsets into the flattened parameter vector
  int oW1, ob1, oW2, ob2, oW3, ob3, ow4, ob4;
};

namespace {
int mfail(qis_mlp* m, int code, const std::string& msg) {
  if (m) m->err = msg;
  else set_global_error(msg.c_str());
  return code;
}
#define MCK(call)                                                                            \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) {                                                                 \
      cudaGetLastError(); /* consume it: a later call must not see this error */              \
      return mfail(m, QIS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));     \
    }                                                                                        \
  } while (0)

template <typename T>
int malloc_m(qis_mlp* m, T** p, size_t count) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), (count ? count : 1) * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return mfail(m, QIS_ERR_OOM, "cudaMalloc failed");
  }
  m->allocs.push_back(*p);
  cudaMemset(*p, 0, (count ? count : 1) * sizeof(T));
  return 0;
}
#define MALLOC(ptr, count)                      \
  do {                                          \
    int rc_ = malloc_m(m, &(ptr), (count));     \
    if (rc_) return rc_;                        \
  } while (0)

template <bool TA, bool TB, typename TBt, bool BR>
void gemm(int M, int N, int K, const float* A, const TBt* B, float* C, const float* bias, int splitk, cudaStream_t s) {
  dim3 g((N + 63) / 64, (M + 63) / 64, splitk);
  k_gemm<TA, TB, TBt, BR><<<g, 256, 0, s>>>(M, N, K, A, B, C, bias);
}

// forward of rows X[0..M) into h1, h2, h3 and z (and loss / dz when y is given)
void mlp_forward(qis_mlp* m, int M, const float* X, const float* y, cudaStream_t s) {
  const int H = m->H;
  gemm<false, false, __nv_bfloat16, true>(M, H, m->F, X, m->Pb + m->oW1, m->h1, m->P + m->ob1, 1, s);
  gemm<false, false, __nv_bfloat16, true>(M, H, H, m->h1, m->Pb + m->oW2, m->h2, m->P + m->ob2, 1, s);
  gemm<false, false, __nv_bfloat16, true>(M, H, H, m->h2, m->Pb + m->oW3, m->h3, m->P + m->ob3, 1, s);
  k_mlp_head<<<(M + 7) / 8, 256, 0, s>>>(M, H, m->h3, m->Pb + m->ow4, m->P + m->ob4, y, m->zb, m->dzb, m->loss,
                                         1.f / (float)M);
}

// gradients of the mean loss over rows X[0..M) into G (zeroed here)
void mlp_backward(qis_mlp* m, int M, const float* X, cudaStream_t s) {
  const int H = m->H;
  cudaMemsetAsync(m->G, 0, sizeof(float) * m->n_params, s);
  const int sk = (M + 511) / 512;                 // split the row reduction of the weight grads
  const int ry = (M + 255) / 256;
  k_head_wgrad<<<dim3((H + 255) / 256, ry), 256, 0, s>>>(M, H, m->h3, m->dzb, m->G + m->ow4);
  k_colsum<<<dim3(1, ry), 32, 0, s>>>(M, 1, m->dzb, m->G + m->ob4);
  k_mlp_head_back<<<(unsigned)(((long long)M * H + 255) / 256), 256, 0, s>>>(M, H, m->dzb, m->Pb + m->ow4, m->h3, m->d1);
  // layer 3: dW3 = h2^T d3, db3 = colsum d3, d2 = d3 W3^T * (h2 > 0)
  gemm<true, false, float, false>(H, H, M, m->h2, m->d1, m->G + m->oW3, nullptr, sk, s);
  k_colsum<<<dim3((H + 255) / 256, ry), 256, 0, s>>>(M, H, m->d1, m->G + m->ob3);
  gemm<false, true, __nv_bfloat16, false>(M, H, H, m->d1, m->Pb + m->oW3, m->d2, nullptr, 1, s);
  k_relu_mask<<<(unsigned)(((long long)M * H + 255) / 256), 256, 0, s>>>((long long)M * H, m->h2, m->d2);
  // layer 2
  gemm<true, false, float, false>(H, H, M, m->h1, m->d2, m->G + m->oW2, nullptr, sk, s);
  k_colsum<<<dim3((H + 255) / 256, ry), 256, 0, s>>>(M, H, m->d2, m->G + m->ob2);
  gemm<false, true, __nv_bfloat16, false>(M, H, H, m->d2, m->Pb + m->oW2, m->d1, nullptr, 1, s);
  k_relu_mask<<<(unsigned)(((long long)M * H + 255) / 256), 256, 0, s>>>((long long)M * H, m->h1, m->d1);
  // layer 1
  gemm<true, false, float, false>(m->F, H, M, X, m->d1, m->G + m->oW1, nullptr, sk, s);
  k_colsum<<<dim3((H + 255) / 256, ry), 256, 0, s>>>(M, H, m->d1, m->G + m->ob1);
}

void refresh_bf16(qis_mlp* m, cudaStream_t s) {
  k_to_bf16<<<(m->n_params + 255) / 256, 256, 0, s>>>(m->n_params, m->P, m->Pb);
}
}  // namespace

extern "C" {

int qis_mlp_create(const qis_mlp_config* cfg, qis_mlp** out) {
  qis_mlp* m = nullptr;
  if (!cfg || !out) return mfail(nullptr, QIS_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (cfg->hidden < 16 || cfg->hidden > 1024 || cfg->hidden % 16) return mfail(nullptr, QIS_ERR_INVALID_ARG, "hidden must be a multiple of 16 in [16, 1024]");
  if (cfg->max_sites < 1 || cfg->batch < 1 || cfg->max_n < 2 || cfg->max_n > kMaxN)
    return mfail(nullptr, QIS_ERR_INVALID_ARG, "bad max_sites / batch / max_n");
  if (cudaSetDevice(cfg->device) != cudaSuccess) return mfail(nullptr, QIS_ERR_CUDA, "cudaSetDevice failed");
  m = new qis_mlp();
  m->cfg = *cfg;
  m->H = cfg->hidden;
  m->cap = cfg->max_sites;
  m->batch = cfg->batch;
  m->max_n = cfg->max_n;
  const int H = m->H, F = m->F;
  m->oW1 = 0;
  m->ob1 = m->oW1 + F * H;
  m->oW2 = m->ob1 + H;
  m->ob2 = m->oW2 + H * H;
  m->oW3 = m->ob2 + H;
  m->ob3 = m->oW3 + H * H;
  m->ow4 = m->ob3 + H;
  m->ob4 = m->ow4 + H;
  m->n_params = m->ob4 + 1;
  auto run = [&]() -> int {
    MCK(cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking));
    MALLOC(m->P, m->n_params);
    MALLOC(m->G, m->n_params);
    MALLOC(m->Mm, m->n_params);
    MALLOC(m->Vv, m->n_params);
    MALLOC(m->Pb, m->n_params);
    MALLOC(m->X, (size_t)m->cap * F);
    MALLOC(m->Y, m->cap);
    const size_t rows = (size_t)std::max(m->batch, m->max_n);
    MALLOC(m->h1, rows * H);
    MALLOC(m->h2, rows * H);
    MALLOC(m->h3, rows * H);
    MALLOC(m->d1, rows * H);
    MALLOC(m->d2, rows * H);
    MALLOC(m->zb, rows);
    MALLOC(m->dzb, rows);
    MALLOC(m->loss, 1);
    MALLOC(m->Jst, (size_t)m->max_n * m->max_n);
    MALLOC(m->hst, m->max_n);
    MALLOC(m->bst, (m->max_n + 63) / 64);
    MALLOC(m->Xq, rows * F);
    // He initialisation from the SplitMix64 stream keyed by the seed (Box-Muller pairs)
    std::vector<float> p(m->n_params, 0.f);
    uint64_t key = splitmix64(cfg->seed ^ 0x4D4C50ull, 0);
    uint64_t c = 0;
    auto gauss = [&]() {
      const double u1 = ((double)(splitmix64(key, c++) >> 11) + 1.0) * 0x1.0p-53;
      const double u2 = (double)(splitmix64(key, c++) >> 11) * 0x1.0p-53;
      return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
    };
    for (int e = 0; e < F * H; ++e) p[m->oW1 + e] = (float)(gauss() * sqrt(2.0 / F));
    for (int e = 0; e < H * H; ++e) p[m->oW2 + e] = (float)(gauss() * sqrt(2.0 / H));
    for (int e = 0; e < H * H; ++e) p[m->oW3 + e] = (float)(gauss() * sqrt(2.0 / H));
    for (int e = 0; e < H; ++e) p[m->ow4 + e] = (float)(gauss() * sqrt(1.0 / H));
    MCK(cudaMemcpy(m->P, p.data(), sizeof(float) * m->n_params, cudaMemcpyHostToDevice));
    refresh_bf16(m, m->stream);
    MCK(cudaStreamSynchronize(m->stream));
    return 0;
  };
  const int rc = run();
  if (rc) {
    set_global_error(m->err.c_str());
    qis_mlp_destroy(m);
    return rc;
  }
  *out = m;
  return 0;
}

void qis_mlp_destroy(qis_mlp* m) {
  if (!m) return;
  cudaSetDevice(m->cfg.device);
  if (m->stream) cudaStreamSynchronize(m->stream);
  for (void* p : m->allocs) cudaFree(p);
  if (m->stream) cudaStreamDestroy(m->stream);
  delete m;
}

const char* qis_mlp_last_error(const qis_mlp* m) { return m ? m->err.c_str() : "NULL network"; }

int qis_mlp_num_params(qis_mlp* m, int* count) {
  if (!m || !count) return mfail(m, QIS_ERR_INVALID_ARG, "NULL argument");
  *count = m->n_params;
  return 0;
}

int qis_mlp_get_params(qis_mlp* m, float* flat) {
  if (!m || !flat) return mfail(m, QIS_ERR_INVALID_ARG, "NULL argument");
  MCK(cudaSetDevice(m->cfg.device));
  MCK(cudaStreamSynchronize(m->stream));
  MCK(cudaMemcpy(flat, m->P, sizeof(float) * m->n_params, cudaMemcpyDeviceToHost));
  return 0;
}

int qis_mlp_set_params(qis_mlp* m, const float* flat) {
  if (!m || !flat) return mfail(m, QIS_ERR_INVALID_ARG, "NULL argument");
  MCK(cudaSetDevice(m->cfg.device));
  MCK(cudaStreamSynchronize(m->stream));
  MCK(cudaMemcpy(m->P, flat, sizeof(float) * m->n_params, cudaMemcpyHostToDevice));
  MCK(cudaMemset(m->Mm, 0, sizeof(float) * m->n_params));
  MCK(cudaMemset(m->Vv, 0, sizeof(float) * m->n_params));
  m->adam_t = 0;
  refresh_bf16(m, m->stream);
  MCK(cudaStreamSynchronize(m->stream));
  return 0;
}

int qis_mlp_features(qis_mlp* m, int n, const double* J, const double* h, float* X_out) {
  if (!m || !J || !h || !X_out) return mfail(m, QIS_ERR_INVALID_ARG, "NULL argument");
  if (n < 2 || n > m->max_n) return mfail(m, QIS_ERR_INVALID_ARG, "n must be in [2, max_n]");
  MCK(cudaSetDevice(m->cfg.device));
  cudaStream_t s = m->stream;
  MCK(cudaMemcpyAsync(m->Jst, J, sizeof(double) * n * n, cudaMemcpyHostToDevice, s));
  MCK(cudaMemcpyAsync(m->hst, h, sizeof(double) * n, cudaMemcpyHostToDevice, s));
  k_mlp_features<<<(n + 127) / 128, 128, 0, s>>>(m->Jst, n, m->hst, n, m->Xq);
  MCK(cudaGetLastError());
  MCK(cudaMemcpyAsync(X_out, m->Xq, sizeof(float) * n * kF, cudaMemcpyDeviceToHost, s));
  MCK(cudaStreamSynchronize(s));
  return 0;
}

int qis_mlp_clear_examples(qis_mlp* m) {
  if (!m) return mfail(m, QIS_ERR_INVALID_ARG, "NULL argument");
  m->n_examples = 0;
  return 0;
}

int qis_mlp_add_example(qis_mlp* m, int n, const double* J, const double* h, const uint64_t* bits) {
  if (!m || !J || !h || !bits) return mfail(m, QIS_ERR_INVALID_ARG, "NULL argument");
  if (n < 2 || n > m->max_n) return mfail(m, QIS_ERR_INVALID_ARG, "n must be in [2, max_n]");
  if (m->n_examples + n > m->cap) return mfail(m, QIS_ERR_CAPACITY, "training set full (max_sites)");
  MCK(cudaSetDevice(m->cfg.device));
  cudaStream_t s = m->stream;
  MCK(cudaMemcpyAsync(m->Jst, J, sizeof(double) * n * n, cudaMemcpyHostToDevice, s));
  MCK(cudaMemcpyAsync(m->hst, h, sizeof(double) * n, cudaMemcpyHostToDevice, s));
  MCK(cudaMemcpyAsync(m->bst, bits, sizeof(uint64_t) * ((n + 63) / 64), cudaMemcpyHostToDevice, s));
  k_mlp_features<<<(n + 127) / 128, 128, 0, s>>>(m->Jst, n, m->hst, n, m->X + (size_t)m->n_examples * kF);
  k_mlp_labels<<<(n + 127) / 128, 128, 0, s>>>(m->bst, n, m->Y + m->n_examples);
  MCK(cudaGetLastError());
  MCK(cudaStreamSynchronize(s));   // staging buffers are reused by the next call
  m->n_examples += n;
  return 0;
}

int qis_mlp_forward(qis_mlp* m, int M, const float* X, float* z_out) {
  if (!m || !X || !z_out || M < 1) return mfail(m, QIS_ERR_INVALID_ARG, "bad argument");
  if (M > std::max(m->batch, m->max_n)) return mfail(m, QIS_ERR_INVALID_ARG, "M exceeds the activation buffers");
  MCK(cudaSetDevice(m->cfg.device));
  cudaStream_t s = m->stream;
  MCK(cudaMemcpyAsync(m->Xq, X, sizeof(float) * M * kF, cudaMemcpyHostToDevice, s));
  mlp_forward(m, M, m->Xq, nullptr, s);
  MCK(cudaGetLastError());
  MCK(cudaMemcpyAsync(z_out, m->zb, sizeof(float) * M, cudaMemcpyDeviceToHost, s));
  MCK(cudaStreamSynchronize(s));
  return 0;
}

int qis_mlp_loss_grad(qis_mlp* m, int M, const float* X, const float* y, double* loss, float* grad_out) {
  if (!m || !X || !y || M < 1) return mfail(m, QIS_ERR_INVALID_ARG, "bad argument");
  if (M > std::max(m->batch, m->max_n)) return mfail(m, QIS_ERR_INVALID_ARG, "M exceeds the activation buffers");
  MCK(cudaSetDevice(m->cfg.device));
  cudaStream_t s = m->stream;
  MCK(cudaMemcpyAsync(m->Xq, X, sizeof(float) * M * kF, cudaMemcpyHostToDevice, s));
  float* ylab = m->d2;   // labels staged in a gradient buffer that is only written after the head
  MCK(cudaMemcpyAsync(ylab, y, sizeof(float) * M, cudaMemcpyHostToDevice, s));
  MCK(cudaMemsetAsync(m->loss, 0, sizeof(double), s));
  mlp_forward(m, M, m->Xq, ylab, s);
  mlp_backward(m, M, m->Xq, s);
  MCK(cudaGetLastError());
  if (loss) MCK(cudaMemcpyAsync(loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
  if (grad_out) MCK(cudaMemcpyAsync(grad_out, m->G, sizeof(float) * m->n_params, cudaMemcpyDeviceToHost, s));
  MCK(cudaStreamSynchronize(s));
  return 0;
}

int qis_mlp_train(qis_mlp* m, int epochs, float lr, double* final_loss) {
  if (!m || epochs < 0 || !(lr > 0)) return mfail(m, QIS_ERR_INVALID_ARG, "bad argument");
  if (m->n_examples < 1) return mfail(m, QIS_ERR_STATE, "no training examples");
  MCK(cudaSetDevice(m->cfg.device));
  cudaStream_t s = m->stream;
  const int N = m->n_examples, Bt = m->batch;
  double last = 0.0;
  for (int ep = 0; ep < epochs; ++ep) {
    MCK(cudaMemsetAsync(m->loss, 0, sizeof(double), s));
    int nb = 0;
    for (int r0 = 0; r0 < N; r0 += Bt, ++nb) {
      const int M = std::min(Bt, N - r0);
      const float* X = m->X + (size_t)r0 * kF;
      mlp_forward(m, M, X, m->Y + r0, s);
      mlp_backward(m, M, X, s);
      ++m->adam_t;
      const float b1 = 0.9f, b2 = 0.999f;
      const float c1 = 1.f - powf(b1, (float)m->adam_t), c2 = 1.f - powf(b2, (float)m->adam_t);
      k_adam<<<(m->n_params + 255) / 256, 256, 0, s>>>(m->n_params, m->P, m->G, m->Mm, m->Vv, lr, b1, b2, 1e-8f, c1, c2);
      refresh_bf16(m, s);
    }
    MCK(cudaGetLastError());
    double sum = 0.0;
    MCK(cudaMemcpyAsync(&sum, m->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    MCK(cudaStreamSynchronize(s));
    last = sum / nb;   // mean of the batch losses of this epoch
  }
  if (final_loss) *final_loss = last;
  return 0;
}

}  // extern "C"

// ---------------------------------------------------------------- warm start of a context
namespace qis {
cudaError_t mlp_propose_states(qis_mlp* m, const double* J64, long long stride, const double* h64, int n, int R,
                               uint64_t key, uint64_t* init_bits, int Wstride, cudaStream_t s) {
  // the network runs on the context's stream; its own stream must be idle
  cudaError_t e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return e;
  k_mlp_features<<<(n + 127) / 128, 128, 0, s>>>(J64, stride, h64, n, m->Xq);
  mlp_forward(m, n, m->Xq, nullptr, s);
  k_mlp_sample<<<dim3(((n + 63) / 64 + 31) / 32, R), 32, 0, s>>>(m->zb, n, R, key, init_bits, Wstride);
  return cudaGetLastError();
}
int mlp_max_n(const qis_mlp* m) { return m->max_n; }
}  // namespace qis
