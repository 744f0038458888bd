// qis_api.cu -- host side of libqis: the C ABI of include/qis.h, context and device memory,
// instance preparation and the iteration driver.
#include <math.h>
#include <stdlib.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "qis_common.cuh"

using namespace qis;

namespace {

std::string g_create_error = "no error";

struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct qis_ctx {
  qis_config cfg{};
  int K1 = 0, R = 0, mode = 0, NP = 0, Wmax = 0, cap = 0, B = 0, max_inst = 0, digit_planes = 0;
  long long pool_mat = 0, pool_vec = 0;
  cudaStream_t stream = nullptr;
  std::vector<InstDesc> inst;
  std::vector<int> inst_ready;  // init_states called
  InstDesc* inst_d = nullptr;
  DevPtrs P{};
  std::vector<void*> allocs;
  // owned (non-const) views of the instance pools
  double* J64 = nullptr;
  double* h64 = nullptr;
  long long* Jq = nullptr;
  float* J4 = nullptr;
  __half* D16 = nullptr;
  int digits_used = 1;     // most digits of any instance (sizes the tensor-core pipeline)
  bool fields_simt = false;  // QIS_FIELDS_SIMT=1: exact int64 SIMT fields instead of tcgen05
  long long* hq = nullptr;
  uint64_t* zob = nullptr;
  double* stats = nullptr;
  double* jstage = nullptr;   // [max_n * max_n] one instance's J as copied from the host (FP64 mode)
  LayoutItem* items_d = nullptr;   // [max_inst] staging places of a creation batch
  uint64_t* all_bits = nullptr;   // [max_inst][K1][Wmax] every instance's merged states
  double* all_E = nullptr;        // [max_inst][K1]
  int4* work = nullptr;    // FP64 scan: 64 x 64 tiles x groups of searches
  int n_work = 0;
  int4* tasks = nullptr;   // FP32 scan: warp tasks (instance, strip, first column, chunk width)
  int n_tasks = 0;
  size_t tasks_cap = 0;
  bool work_dirty = true;
  bool merged_fresh = false;
  std::vector<char> init_pending;  // instance whose searches wait for their start (one launch for all)
  // initial states given by the host: held here until the searches start, then uploaded in one
  // copy per run of consecutive instances (instead of one small copy per call)
  std::vector<uint64_t> init_host;   // [max_inst * R][Wmax]
  std::vector<char> init_from_host;  // instance whose initial states wait in init_host
  // init_E / init_q hold the energies of the instance's current initial states (formed by
  // k_init_energy or k_init_search; the fused search kernel's deferred values do not count here:
  // a run that failed may have formed them from bad fields)
  std::vector<char> e0_valid;
  // instances whose searches were started with their initial energies left to the fused search
  // kernel, and whether that kernel has not been enqueued yet (the call failed before it): such
  // instances are started again, energies included, by the next entry point
  std::vector<char> e0_deferred;
  bool e0_unresolved = false;
  bool counts_valid = false;      // mrg_counts holds the counts of the current merge (status checked)
  std::vector<int> mrg_counts;
  uint64_t* scratch_bits = nullptr;  // [kScratch][Wmax]
  double* scratch_E = nullptr;
  int scratch_states = 0;
  uint64_t launches = 0;
  uint64_t cand_acc[2] = {0, 0};  // candidates of instances removed by qis_clear_instances
  // tunables (results never depend on them): scan chunk width 32 * tune_nc columns, searches
  // per scan task (0 = all R of the instance), searches per GEMM tile (0 = automatic)
  qis_tuning tune{8, 0, 0, 0};
  // kernel timing (qis_profile_*): per class, event pairs recorded since the last query
  bool profiling = false;
  bool use_graph = true;                    // QIS_NO_GRAPH=1 launches the kernels one by one
  bool no_fused = false;                    // QIS_FUSED=0: the per-kernel form of every iteration
  cudaGraphExec_t graph_exec = nullptr;     // one iteration, captured for the current instances
  int graph_n = 0;                          // fused form: the iteration count the graph was captured for
  int last_n = 0;                           // fused form: the iteration count of the previous call
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[8];
  size_t ev_used[8] = {0};
  std::string err = "no error";
};

namespace {

int fail(qis_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  else g_create_error = msg;
  return code;
}

// On failure the runtime's last-error state is consumed, so a later call does not report it.
#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) {                                                                  \
      cudaGetLastError();                                                                     \
      return fail(ctx, QIS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));     \
    }                                                                                         \
  } while (0)

#define LAUNCH(call)                                                                          \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    ++ctx->launches;                                                                          \
    if (e_ != cudaSuccess) {                                                                  \
      cudaGetLastError();                                                                     \
      return fail(ctx, QIS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));     \
    }                                                                                         \
  } while (0)

template <typename T>
int dalloc(qis_ctx* ctx, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, QIS_ERR_OOM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
  }
  ctx->allocs.push_back(*p);
  cudaMemset(*p, 0, count * sizeof(T));
  return 0;
}

#define ALLOC(ptr, count)                     \
  do {                                        \
    int rc_ = dalloc(ctx, &(ptr), (count));   \
    if (rc_) return rc_;                      \
  } while (0)

// Key of the library's initial-state stream for instance `id` (SplitMix64 chain).
uint64_t state_key(uint64_t seed, int id) {
  uint64_t k = splitmix64(seed, 0);
  k = splitmix64(k ^ (uint64_t)id, 0);
  k = splitmix64(k ^ 3ull, 0);
  return k;
}

int check_status(qis_ctx* ctx) {
  int st = 0;
  CK(cudaMemcpy(&st, ctx->P.status, sizeof(int), cudaMemcpyDeviceToHost));
  // a timeout first: the kernels after a timed-out one run on fields it did not write, so any
  // other flag they raise is a consequence
  if (st & kStatTimeout)
    return fail(ctx, QIS_ERR_DEVICE_TIMEOUT,
                "a bounded device-side wait gave up; the searches are undefined until qis_reset");
  if (st & kStatCapacity)
    return fail(ctx, QIS_ERR_CAPACITY,
                "a search produced more survivors than survivor_cap (raise survivor_cap); the searches are "
                "undefined until qis_reset");
  if (st) return fail(ctx, QIS_ERR_STATE, "device reported an inconsistent search state");
  return 0;
}

int sync_and_check(qis_ctx* ctx) {
  CK(cudaStreamSynchronize(ctx->stream));
  return check_status(ctx);
}

// Candidates of the current instances: every productive iteration of a search of an n-spin
// instance evaluates n(n-1)/2 pairs and n singles.
int count_candidates(qis_ctx* ctx, uint64_t c[2]) {
  c[0] = c[1] = 0;
  if (ctx->P.B == 0) return 0;
  std::vector<int> np(ctx->P.B);
  CK(cudaMemcpy(np.data(), ctx->P.nprod, sizeof(int) * np.size(), cudaMemcpyDeviceToHost));
  std::vector<unsigned long long> pp(ctx->P.B);
  CK(cudaMemcpy(pp.data(), ctx->P.npair, sizeof(unsigned long long) * pp.size(), cudaMemcpyDeviceToHost));
  for (size_t id = 0; id < ctx->inst.size(); ++id) {
    const uint64_t n = (uint64_t)ctx->inst[id].n;
    uint64_t it = 0;
    for (int r = 0; r < ctx->R; ++r) {
      const size_t b = (size_t)ctx->inst[id].first_search + r;
      it += (uint64_t)np[b];
      c[0] += pp[b];
    }
    if (ctx->cfg.flips != QIS_FLIPS_EXCHANGE) c[1] += it * n;
  }
  return 0;
}

// Record the start event of a timed launch of class `k` (no-op unless profiling).
cudaError_t prof_begin(qis_ctx* ctx, int k) {
  if (!ctx->profiling) return cudaSuccess;
  auto& v = ctx->ev[k];
  if (ctx->ev_used[k] == v.size()) {
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&b);
    if (e != cudaSuccess) return e;
    v.emplace_back(a, b);
  }
  return cudaEventRecord(v[ctx->ev_used[k]].first, ctx->stream);
}

cudaError_t prof_end(qis_ctx* ctx, int k) {
  if (!ctx->profiling) return cudaSuccess;
  cudaError_t e = cudaEventRecord(ctx->ev[k][ctx->ev_used[k]].second, ctx->stream);
  ++ctx->ev_used[k];
  return e;
}

// The five kernels of one iteration of Alg. 3 (each bracketed by timing events when profiling).
// The output-sensitive pair scan runs in the split modes up to a padded size of 4096 (its
// per-search shared-memory arrays), by default or when asked for; the dense tiles otherwise.
static bool sparse_allowed(const qis_ctx* ctx) { return ctx->mode != QIS_FP64 && ctx->NP <= kSparseMaxNP; }
static bool sparse_scan(const qis_ctx* ctx) { return sparse_allowed(ctx) && ctx->tune.pair_scan != 2; }
// The fused search kernel: the output-sensitive scan (pair_scan 0 or 1) with fields by update,
// a padded n and a list small enough for its shared-memory arrays (QIS_FUSED=0 turns it off).
static bool fused_search(const qis_ctx* ctx) {
  return sparse_scan(ctx) && ctx->tune.pair_scan != 3 && ctx->NP <= kSearchMaxNP && ctx->K1 <= kSearchMaxK1 &&
         ctx->P.inc_on && !ctx->fields_simt && !ctx->no_fused;
}

// Every iteration of a qis_iterate call in one launch of the fused search kernel: the first
// iteration's parent pick and fields run first as their own kernels (the tensor-core GEMM
// computes the fields of every parent without a stored generator, e.g. every initial state),
// then one block per search runs its n iterations.
int launch_iterations_fused(qis_ctx* ctx, int n, cudaStream_t s) {
  ctx->P.dense_ctl = 0;
  const DevPtrs& P = ctx->P;
  CK(prof_begin(ctx, 0));
  LAUNCH(launch_pick(P, s));
  CK(prof_end(ctx, 0));
  CK(prof_begin(ctx, 1));
  LAUNCH(launch_fields_inc(P, s));
  LAUNCH(launch_fields_tc(P, ctx->D16, P.S16, ctx->max_inst, ctx->digits_used, P.gemm_nt, s));
  CK(prof_end(ctx, 1));
  CK(prof_begin(ctx, 5));
  LAUNCH(launch_search(P, n, s));
  CK(prof_end(ctx, 5));
  return 0;
}

int launch_iteration(qis_ctx* ctx, cudaStream_t s) {
  ctx->P.dense_ctl = !sparse_scan(ctx);   // the output-sensitive scan reads no control words
  const DevPtrs& P = ctx->P;
  CK(prof_begin(ctx, 0));
  LAUNCH(launch_pick(P, s));
  CK(prof_end(ctx, 0));
  CK(prof_begin(ctx, 1));
  if (P.inc_on) LAUNCH(launch_fields_inc(P, s));   // the rest: tiles the GEMM computes in full
  if (ctx->mode == QIS_FP64) LAUNCH(launch_fields_fp64(P, s));
  else if (ctx->fields_simt) LAUNCH(launch_fields_exact(P, s));
  else LAUNCH(launch_fields_tc(P, ctx->D16, P.S16, ctx->max_inst, ctx->digits_used, P.gemm_nt, s));
  CK(prof_end(ctx, 1));
  CK(prof_begin(ctx, 2));
  LAUNCH(launch_bound(P, s));
  CK(prof_end(ctx, 2));
  CK(prof_begin(ctx, 3));
  if (ctx->cfg.flips == QIS_FLIPS_SINGLE) {
    // no pair candidates: nothing to scan
  } else if (ctx->mode == QIS_FP64) {
    LAUNCH(launch_scan64(P, ctx->work, ctx->n_work, s));
  } else if (sparse_scan(ctx)) {
    LAUNCH(launch_scan_sparse(P, s));   // output-sensitive: work proportional to the survivors
  } else {
    LAUNCH(launch_scan_pairs(P, ctx->tasks, ctx->n_tasks, ctx->tune.scan_search_group > 0 ? ctx->tune.scan_search_group : ctx->R, s));
  }
  CK(prof_end(ctx, 3));
  CK(prof_begin(ctx, 4));
  LAUNCH(launch_merge(P, s));
  CK(prof_end(ctx, 4));
  return 0;
}

void drop_graph(qis_ctx* ctx) {
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  ctx->graph_exec = nullptr;
  ctx->graph_n = 0;
  ctx->last_n = 0;
}

int build_work(qis_ctx* ctx) {
  // searches per tensor-core tile: also the tiling of the spin operand that k_pick writes
  ctx->P.gemm_nt = ctx->tune.gemm_tile_searches > 0 ? ctx->tune.gemm_tile_searches
                                                      : gemm_tile_n(ctx->R, ctx->digits_used);
  std::vector<int4> w;
  for (int id = 0; id < (int)ctx->inst.size() && ctx->mode == QIS_FP64; ++id) {   // the FP64 scan's tiles
    const int nb = (ctx->inst[id].n + kTile - 1) / kTile;
    for (int bi = 0; bi < nb; ++bi)
      for (int bj = bi; bj < nb; ++bj)
        for (int g = 0; g * kScan64Group < ctx->R; ++g) w.push_back(make_int4(id, bi, bj, g));
  }
  ctx->n_work = (int)w.size();
  const size_t cap_items = (size_t)ctx->max_inst * ((ctx->NP / kTile) * (ctx->NP / kTile + 1) / 2) *
                           ((ctx->R + kScan64Group - 1) / kScan64Group);
  if (w.size() > cap_items) return fail(ctx, QIS_ERR_STATE, "work list overflow");
  if (!w.empty()) CK(cudaMemcpyAsync(ctx->work, w.data(), w.size() * sizeof(int4), cudaMemcpyHostToDevice, ctx->stream));
  // warp tasks of the FP32 pair scan, widest chunks first (better tail balance)
  std::vector<int4> t;
  const int RG = ctx->tune.scan_search_group > 0 ? ctx->tune.scan_search_group : ctx->R;
  const bool dense = ctx->mode != QIS_FP64 && !sparse_scan(ctx);   // only the dense FP32 scan reads them
  for (int id = 0; id < (int)ctx->inst.size() && dense; ++id)
    scan_tasks_for(id, ctx->inst[id].n, ctx->tune.scan_chunk_nc, ctx->R, RG, t);
  std::stable_sort(t.begin(), t.end(), [](const int4& a, const int4& b) { return (a.w & 0xff) > (b.w & 0xff); });
  if (t.size() > ctx->tasks_cap)
    return fail(ctx, QIS_ERR_INVALID_ARG, "too many scan tasks for this tuning (wider chunks or larger search groups)");
  ctx->n_tasks = (int)t.size();
  // (copies from pageable memory: the host vectors are free once the calls return)
  if (!t.empty()) CK(cudaMemcpyAsync(ctx->tasks, t.data(), t.size() * sizeof(int4), cudaMemcpyHostToDevice, ctx->stream));
  ctx->work_dirty = false;
  return 0;
}

}  // namespace

void qis::set_global_error(const char* msg) { g_create_error = msg; }

extern "C" {

int qis_create(const qis_config* cfg, qis_ctx** out) {
  qis_ctx* ctx = nullptr;
  if (!cfg || !out) return fail(nullptr, QIS_ERR_INVALID_ARG, "cfg and out must not be NULL");
  *out = nullptr;
  if (cfg->K < 1 || cfg->K + 1 > 4096) return fail(nullptr, QIS_ERR_INVALID_ARG, "K must satisfy 1 <= K and K+1 <= 4096");
  if (cfg->R < 1 || cfg->R > 65536) return fail(nullptr, QIS_ERR_INVALID_ARG, "R must be in [1, 65536]");
  if (cfg->max_n < 2 || cfg->max_n > kMaxN) return fail(nullptr, QIS_ERR_INVALID_ARG, "max_n must be in [2, 16384]");
  if (cfg->max_instances < 1) return fail(nullptr, QIS_ERR_INVALID_ARG, "max_instances must be >= 1");
  if (cfg->precision != QIS_FP64 && cfg->precision != QIS_SPLIT_BF16 && cfg->precision != QIS_PM1_FP8)
    return fail(nullptr, QIS_ERR_INVALID_ARG, "unknown precision mode");
  if (cfg->flips < QIS_FLIPS_SINGLE_PAIR || cfg->flips > QIS_FLIPS_EXCHANGE)
    return fail(nullptr, QIS_ERR_INVALID_ARG, "unknown flip set");
  int cap = cfg->survivor_cap ? cfg->survivor_cap : 2048;
  if (cap < 4 * (cfg->K + 1) + 64 || cap > 16384)
    return fail(nullptr, QIS_ERR_INVALID_ARG, "survivor_cap must be in [4(K+1)+64, 16384]");
  {
    cudaError_t e = cudaSetDevice(cfg->device);
    if (e != cudaSuccess) return fail(nullptr, QIS_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  }
  ctx = new qis_ctx();
  ctx->cfg = *cfg;
  ctx->K1 = cfg->K + 1;
  ctx->R = cfg->R;
  ctx->mode = cfg->precision;
  ctx->NP = pad_of(cfg->max_n);
  ctx->Wmax = words_of(cfg->max_n);
  ctx->cap = cap;
  ctx->max_inst = cfg->max_instances;
  ctx->B = cfg->max_instances * cfg->R;
  ctx->pool_mat = (long long)ctx->max_inst * ctx->NP * ctx->NP;
  ctx->pool_vec = (long long)ctx->max_inst * ctx->NP;
  ctx->digit_planes = (ctx->mode == QIS_FP64) ? 0 : (ctx->mode == QIS_PM1_FP8 ? 1 : kMaxDigits);
  {
    const char* e = getenv("QIS_FIELDS_SIMT");
    ctx->fields_simt = e && e[0] == '1';
    const char* ds = getenv("QIS_DENSE_SCAN");
    if (ds && ds[0] == '1') ctx->tune.pair_scan = 2;   // the register-tile pair scan by default
    const char* g = getenv("QIS_NO_GRAPH");
    ctx->use_graph = !(g && g[0] == '1');
    const char* fz = getenv("QIS_FUSED");
    ctx->no_fused = fz && fz[0] == '0';
  }
  auto bail = [&](int rc) {
    g_create_error = ctx->err;
    qis_destroy(ctx);
    return rc;
  };
  int rc = 0;
  auto run = [&]() -> int {
    CK(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
    const size_t B = ctx->B, K1 = ctx->K1, W = ctx->Wmax, NP = ctx->NP;
    InstDesc* id = nullptr;
    ALLOC(id, ctx->max_inst);
    ctx->inst_d = id;
    ALLOC(ctx->J64, ctx->pool_mat);
    ALLOC(ctx->h64, ctx->pool_vec);
    if (ctx->mode != QIS_FP64) {
      ALLOC(ctx->Jq, ctx->pool_mat);
      ALLOC(ctx->J4, ctx->pool_mat);
      ALLOC(ctx->D16, (size_t)ctx->digit_planes * ctx->pool_mat);
      ALLOC(ctx->hq, ctx->pool_vec);
    }
    ALLOC(ctx->zob, kMaxN);
    ALLOC(ctx->stats, (size_t)ctx->max_inst * (NP + 8));   // validation statistics of every instance
    ALLOC(ctx->items_d, (size_t)ctx->max_inst);
    if (ctx->mode == QIS_FP64) ALLOC(ctx->jstage, (size_t)cfg->max_n * cfg->max_n);   // the split modes stage in Jq
    ALLOC(ctx->all_bits, (size_t)ctx->max_inst * K1 * W);
    ALLOC(ctx->all_E, (size_t)ctx->max_inst * K1);
    ALLOC(ctx->work, (size_t)ctx->max_inst * ((NP / kTile) * (NP / kTile + 1) / 2) *
                         ((ctx->R + kScan64Group - 1) / kScan64Group));
    ctx->tasks_cap = (size_t)ctx->max_inst * (NP / 8) * (NP / 32 + 2);
    ALLOC(ctx->tasks, ctx->tasks_cap);
    DevPtrs& P = ctx->P;
    P.inst = ctx->inst_d;
    P.n_inst = 0;
    P.R = ctx->R;
    P.K1 = ctx->K1;
    P.Wmax = ctx->Wmax;
    P.cap = ctx->cap;
    P.mode = ctx->mode;
    P.B = 0;
    P.NP = ctx->NP;
    P.flips = ctx->cfg.flips;
    P.wait_ns = 2000000000ull;
    P.wait_probe = 0;
    P.J64 = ctx->J64;
    P.Jq = ctx->Jq;
    P.J4 = ctx->J4;
    P.D16 = ctx->D16;
    P.pool_mat = ctx->pool_mat;
    P.h64 = ctx->h64;
    P.hq = ctx->hq;
    P.zob = ctx->zob;
    ALLOC(P.lst_bits, B * K1 * W);
    ALLOC(P.lst_E, B * K1);
    ALLOC(P.lst_q, B * K1);
    ALLOC(P.lst_key, B * K1);
    ALLOC(P.lst_stamp, B * K1);
    ALLOC(P.lst_hash, B * K1);
    ALLOC(P.lst_used, B * K1);
    ALLOC(P.lst_ord, B * K1);
    ALLOC(P.lst_count, B);
    ALLOC(P.par_bits, B * W);
    ALLOC(P.par_E, B);
    ALLOC(P.par_q, B);
    ALLOC(P.par_hash, B);
    ALLOC(P.active, B);
    ALLOC(P.iter_t, B);
    ALLOC(P.par_stamp, B);
    ALLOC(P.ring_t0, B);
    ALLOC(P.full_tile, (size_t)ctx->max_inst * ((ctx->R + 15) / 16));
    P.ring_n = 1;
    P.ring_slot = (long long)B * NP;
    if (ctx->mode != QIS_FP64) {
      // the exact fields of the last ring_n parents of every search (fields by update): as many
      // iterations as fit in 4 GiB, 2 .. 128 (QIS_FIELD_RING overrides)
      const size_t slot = (size_t)B * NP * sizeof(long long);
      int rn = (int)std::min<size_t>(128, std::max<size_t>(2, (4ull << 30) / slot));
      const char* e = getenv("QIS_FIELD_RING");
      if (e && atoi(e) >= 2) rn = atoi(e);
      P.ring_n = rn;
      P.inc_on = ctx->fields_simt ? 0 : 1;
      ALLOC(P.aq, (size_t)rn * B * NP);
      ALLOC(P.as32, B * NP);
      P.s16_stride = (long long)(ctx->R + 255) * NP;   // room for ceil(R / NT) tiles of any NT <= 256
      ALLOC(P.S16, (size_t)ctx->max_inst * P.s16_stride);
    } else {
      ALLOC(P.a64, B * NP);
      ALLOC(P.amin64, B);
    }
    ALLOC(P.thr32, B);
    ALLOC(P.amin32, B);
    if (ctx->mode != QIS_FP64) ALLOC(P.rm4, (size_t)ctx->pool_vec);
    if (ctx->mode != QIS_FP64) {
      ALLOC(P.sctl, B * (size_t)(NP / 32));
    }
    ALLOC(P.thrE, B);
    ALLOC(P.capE, B);
    ALLOC(P.surv_cnt, B);
    ALLOC(P.dup_c, (size_t)B * K1);
    ALLOC(P.dup_n, B);
    ALLOC(P.surv, B * (size_t)ctx->cap);
    {
      size_t pc = 256;
      while (pc < (size_t)ctx->cap) pc <<= 1;
      ALLOC(P.mrg_scratch, B * 2 * pc);
      P.merge_cand = 512;
      const char* e = getenv("QIS_MERGE_SMEM_CAND");
      if (e) {
        const int v = atoi(e);
        if (v >= 32 && v <= 512 && (v & (v - 1)) == 0) P.merge_cand = v;
      }
    }
    ALLOC(P.init_bits, B * W);
    ALLOC(P.init_E, B);
    ALLOC(P.init_q, B);
    ALLOC(P.e0_pend, B);
    CK(cudaMemset(P.e0_pend, 0, sizeof(int) * B));
    ALLOC(P.status, 4);
    ALLOC(P.nprod, B);
    ALLOC(P.npair, B);
    ALLOC(P.eval_cnt, 64);
    ALLOC(P.surv_tot, 64);
    ALLOC(P.mrg_ref, (size_t)ctx->max_inst * K1);
    ALLOC(P.mrg_src, (size_t)ctx->max_inst * K1);
    ALLOC(P.mrg_count, ctx->max_inst);
    ctx->scratch_states = 4096;
    ALLOC(ctx->scratch_bits, (size_t)ctx->scratch_states * W);
    ALLOC(ctx->scratch_E, ctx->scratch_states);
    {   // partial energy sums of the rescoring when a state group's rows are split over blocks
      size_t m = std::max<size_t>((size_t)ctx->max_inst * K1, (size_t)B);
      m = std::max<size_t>(m, (size_t)ctx->scratch_states);
      ALLOC(P.rs_acc, 2 * m * 32);   // [state][row part][2], at most 32 parts
      int sms = 0;
      CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->cfg.device));
      P.sms = sms;
    }
    // Zobrist keys of the sites (SplitMix64 stream with a fixed key)
    std::vector<uint64_t> z(kMaxN);
    for (int i = 0; i < kMaxN; ++i) z[i] = splitmix64(0x2F0A7B6C5D4E3F21ull, (uint64_t)i);
    CK(cudaMemcpy(ctx->zob, z.data(), kMaxN * sizeof(uint64_t), cudaMemcpyHostToDevice));
    // kernel attributes for the large dynamic shared-memory users
    CK(cudaDeviceSynchronize());
    return 0;
  };
  rc = run();
  if (rc) return bail(rc);
  *out = ctx;
  return 0;
}

void qis_destroy(qis_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->cfg.device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (auto& v : ctx->ev)
    for (auto& pr : v) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  for (void* p : ctx->allocs) cudaFree(p);
  drop_graph(ctx);
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

const char* qis_last_error(const qis_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

namespace {

// Argument checks of one instance that is to become id `id`.
int check_instance_args(qis_ctx* ctx, int id, int n, const double* J, const double* h) {
  if (!J || !h) return fail(ctx, QIS_ERR_INVALID_ARG, "J and h must not be NULL");
  if (n < 2 || n > ctx->cfg.max_n) return fail(ctx, QIS_ERR_INVALID_ARG, "n must be in [2, max_n]");
  if (id >= ctx->max_inst) return fail(ctx, QIS_ERR_INVALID_ARG, "instance table full");
  if (n < 63 && (uint64_t)ctx->cfg.K >= (1ull << n))
    return fail(ctx, QIS_ERR_INVALID_ARG, "K must be below 2^n (Alg. 2 requires 1 <= K < 2^N)");
  return 0;
}

// Copy J of instance id to the device (asynchronous on the library stream) as one contiguous
// block (a pitched copy from pageable memory goes row by row), into `stage`.
int copy_instance(qis_ctx* ctx, int n, const double* J, double* stage) {
  CK(cudaMemcpyAsync(stage, J, sizeof(double) * (size_t)n * n, cudaMemcpyHostToDevice, ctx->stream));
  return 0;
}

// The device address of page-locked host memory at p (registered or allocated by CUDA, so the
// GPU reads it over the host link), or NULL for any other memory.
const double* pinned_view(const double* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();   // not a sticky error: clear it and stage the copy
    return nullptr;
  }
  if (a.type == cudaMemoryTypeHost && a.devicePointer) return reinterpret_cast<const double*>(a.devicePointer);
  return nullptr;
}

// h of instances first .. first+count-1, zero padded to NP, in one copy (their regions are
// consecutive). A copy from pageable memory has left `hall` once it returns.
int copy_fields_h(qis_ctx* ctx, int first, int count, const int* n, const double* const* h) {
  std::vector<double> hall((size_t)count * ctx->NP, 0.0);
  for (int k = 0; k < count; ++k) memcpy(hall.data() + (size_t)k * ctx->NP, h[k], sizeof(double) * n[k]);
  CK(cudaMemcpyAsync(ctx->h64 + (long long)first * ctx->NP, hall.data(), sizeof(double) * hall.size(),
                     cudaMemcpyHostToDevice, ctx->stream));
  return 0;
}

// The padded layout of instance id's J from `stage`, and its validation into stats slot `slot`.
int lay_out_instance(qis_ctx* ctx, int id, int slot, int n, const double* stage) {
  const long long off_mat = (long long)id * ctx->NP * ctx->NP, off_vec = (long long)id * ctx->NP;
  cudaStream_t s = ctx->stream;
  LAUNCH(launch_restride(stage, n, pad_of(n), ctx->J64 + off_mat, s));
  LAUNCH(launch_validate(ctx->P, id, n, off_mat, off_vec, ctx->stats + (size_t)slot * (ctx->NP + 8), s));
  return 0;
}

// The descriptor of instance id from its validation statistics (host): the checks of J and
// h, the fixed-point grid 2^-q and the number of base-4096 digits.
int describe_instance(qis_ctx* ctx, int id, int n, const double* st, InstDesc& d) {
  d = InstDesc{};
  d.n = n;
  d.n_pad = pad_of(n);
  d.W = words_of(n);
  d.first_search = id * ctx->R;
  d.off_mat = (long long)id * ctx->NP * ctx->NP;
  d.off_vec = (long long)id * ctx->NP;
  int bad, maxfrac;
  uint64_t mjb, mhb;
  memcpy(&bad, &st[0], sizeof(int));
  memcpy(&maxfrac, &st[1], sizeof(int));
  memcpy(&mjb, &st[2], 8);
  memcpy(&mhb, &st[3], 8);
  double maxJ, maxh;
  memcpy(&maxJ, &mjb, 8);
  memcpy(&maxh, &mhb, 8);
  if (bad & 1) return fail(ctx, QIS_ERR_INVALID_ARG, "J contains NaN or Inf");
  if (bad & 8) return fail(ctx, QIS_ERR_INVALID_ARG, "h contains NaN or Inf");
  if (bad & 2) return fail(ctx, QIS_ERR_INVALID_ARG, "J has a nonzero diagonal entry");
  if (bad & 4) return fail(ctx, QIS_ERR_INVALID_ARG, "J is not symmetric");
  d.q = -1;
  d.digits = 0;
  d.inv_scale = 1.0;
  d.rounded = 0;
  d.j4max = 0.f;
  d.j4max64 = 4.0 * maxJ;   // exact (power-of-two scaling)
  if (ctx->mode != QIS_FP64) {
    double S = 0.0;
    for (int i = 0; i < n; ++i) S += st[4 + i];
    S += st[4 + n];
    int qmax = 51;
    if (S > 0) qmax = 51 - (int)floor(log2(S));
    int q = maxfrac;
    if (ctx->mode == QIS_PM1_FP8) {
      if (maxfrac != 0 || maxJ > 15.0)
        return fail(ctx, QIS_ERR_INVALID_ARG, "QIS_PM1_FP8 needs integer J with |J_ij| <= 15 and integer h");
      if (qmax < 0) return fail(ctx, QIS_ERR_INVALID_ARG, "energies exceed 2^52");
      q = 0;
    } else if (q > qmax) {
      q = qmax;
      d.rounded = 1;
    }
    if (q < 0) return fail(ctx, QIS_ERR_INVALID_ARG, "couplings too large for exact 64-bit energies");
    const double maxJq = ldexp(maxJ, q);
    const int dbits = (d.n_pad <= 8192) ? 12 : 11;   // exact FP32 partial sums of the digit GEMM
    int digits = 1;
    while (digits < kMaxDigits && ldexp(1.0, dbits * digits - 1) <= maxJq + 0.5) ++digits;
    if (ldexp(1.0, dbits * digits - 1) <= maxJq + 0.5) return fail(ctx, QIS_ERR_INVALID_ARG, "coupling range too wide");
    d.dbits = dbits;
    if (ctx->mode == QIS_PM1_FP8) digits = 1;
    d.q = q;
    d.digits = digits;
    d.inv_scale = ldexp(1.0, -q);
    d.j4max = (float)(4.0 * ldexp(rint(maxJq), -q)) * (1.0f + 1e-6f);
  }
  return 0;
}

// Register described instances ids first .. first+count-1: descriptors to the device, the
// fixed-point planes, the host tables (asynchronous on the library stream).
int register_instances(qis_ctx* ctx, int first, const std::vector<InstDesc>& ds) {
  cudaStream_t s = ctx->stream;
  CK(cudaMemcpyAsync(ctx->inst_d + first, ds.data(), sizeof(InstDesc) * ds.size(), cudaMemcpyHostToDevice, s));
  if (ctx->mode != QIS_FP64 && !ds.empty()) {
    // fixed-point planes, digits and row maxima of the whole batch: two launches
    int max_pad = 0;
    for (const InstDesc& d : ds) max_pad = std::max(max_pad, d.n_pad);
    LAUNCH(launch_prepare_batch(ctx->P, first, (int)ds.size(), max_pad, ctx->D16, ctx->Jq, ctx->J4, ctx->hq, s));
  }
  for (size_t k = 0; k < ds.size(); ++k) {
    const InstDesc& d = ds[k];
    ctx->inst.push_back(d);
    if (d.digits > ctx->digits_used) ctx->digits_used = d.digits;
    ctx->inst_ready.push_back(0);
    ctx->init_pending.push_back(0);
    ctx->init_from_host.push_back(0);
    ctx->e0_valid.push_back(0);
    ctx->e0_deferred.push_back(0);
  }
  ctx->P.n_inst = (int)ctx->inst.size();
  ctx->P.B = ctx->P.n_inst * ctx->R;
  ctx->work_dirty = true;
  drop_graph(ctx);
  ctx->merged_fresh = false;
  return 0;
}

}  // namespace

namespace {

// Start (Alg. 3: the initial state as the only list entry) every search whose instance got new
// initial states, or was reset, since the last flush: one launch per run of consecutive such
// instances. Called first by every entry point that reads or changes the searches.
// defer (qis_iterate, when the fused search kernel runs at least one iteration): the initial
// energies of the split modes are not computed here; the kernel forms them from the exact fields
// of the first iteration (E = (sum_i s_i f_i + sum_i s_i h_i) / 2), which the tensor-core GEMM
// computes for every initial state anyway. Otherwise they come from k_init_energy, or from
// init_E / init_q when those still hold them.
int flush_init(qis_ctx* ctx, bool defer) {
  const int ni = (int)ctx->init_pending.size();
  if (ctx->e0_unresolved) {   // a deferred start whose kernel never ran: start those again
    for (int x = 0; x < ni; ++x)
      if (ctx->e0_deferred[x]) ctx->init_pending[x] = 1;
    ctx->e0_unresolved = false;
  }
  std::fill(ctx->e0_deferred.begin(), ctx->e0_deferred.end(), 0);
  for (int a = 0; a < ni;) {
    if (!ctx->init_pending[a]) {
      ++a;
      continue;
    }
    int e = a;
    while (e < ni && ctx->init_pending[e]) ctx->init_pending[e++] = 0;
    // the host-given initial states of the range: one copy per run of such instances
    for (int x = a; x < e;) {
      if (!ctx->init_from_host[x]) {
        ++x;
        continue;
      }
      int y = x;
      while (y < e && ctx->init_from_host[y]) ctx->init_from_host[y++] = 0;
      const size_t off = (size_t)ctx->inst[x].first_search * ctx->Wmax;
      const size_t len = (size_t)(y - x) * ctx->R * ctx->Wmax;
      CK(cudaMemcpyAsync(ctx->P.init_bits + off, ctx->init_host.data() + off, len * sizeof(uint64_t),
                         cudaMemcpyHostToDevice, ctx->stream));
      x = y;
    }
    // split modes: the initial energies of the range in groups of states per block first
    // (unless they are known or deferred); FP64 mode: formed by k_init_search itself
    const bool grouped = ctx->mode != QIS_FP64;
    bool known = true;
    for (int x = a; x < e; ++x) known = known && ctx->e0_valid[x];
    const bool deferred = grouped && defer && !known;
    if (deferred) {
      for (int x = a; x < e; ++x) ctx->e0_deferred[x] = 1;
      ctx->e0_unresolved = true;
    } else if (grouped && !known) {
      int max_n = 0;
      for (int x = a; x < e; ++x) max_n = std::max(max_n, ctx->inst[x].n);
      LAUNCH(launch_init_energy(ctx->P, a, e - a, max_n, ctx->stream));
    }
    LAUNCH(launch_init_search(ctx->P, ctx->inst[a].first_search, (e - a) * ctx->R, ctx->stream,
                              known || (grouped && !deferred), deferred));
    if (!deferred)
      for (int x = a; x < e; ++x) ctx->e0_valid[x] = 1;
    a = e;
  }
  return 0;
}

}  // namespace

#define FLUSH_INIT(ctx)                     \
  do {                                      \
    const int rc_ = flush_init(ctx, false); \
    if (rc_) return rc_;                    \
  } while (0)

int qis_create_instance(qis_ctx* ctx, int n, const double* J, const double* h, int* instance_id) {
  const double* Jp[1] = {J};
  const double* hp[1] = {h};
  return qis_create_instances(ctx, 1, &n, Jp, hp, instance_id);
}

int qis_create_instances(qis_ctx* ctx, int count, const int* n, const double* const* J, const double* const* h,
                         int* instance_ids) {
  if (!ctx) return fail(nullptr, QIS_ERR_INVALID_ARG, "ctx is NULL");
  if (count < 0 || (count > 0 && (!n || !J || !h))) return fail(ctx, QIS_ERR_INVALID_ARG, "bad arrays");
  if (count == 0) return 0;
  const int first = (int)ctx->inst.size();
  for (int k = 0; k < count; ++k) {
    const int rc = check_instance_args(ctx, first + k, n[k], J[k], h[k]);
    if (rc) return rc;
  }
  CK(cudaSetDevice(ctx->cfg.device));
  // every copy, then every layout and validation, then one read-back of all statistics. In the
  // split modes each instance is staged in its own region of the fixed-point pool (written
  // from J64 later), so the copies run back to back; the FP64 mode stages one instance at a
  // time (a copy from pageable memory first waits for the stream, so the buffer is free again).
  {
    const int rc = copy_fields_h(ctx, first, count, n, h);
    if (rc) return rc;
  }
  if (ctx->mode != QIS_FP64) {
    // a page-locked J is read by the layout kernel itself (one pass over the host memory);
    // any other J is staged with a copy first
    std::vector<const double*> src(count);
    for (int k = 0; k < count; ++k) {
      src[k] = pinned_view(J[k]);
      if (src[k]) continue;
      double* stage = reinterpret_cast<double*>(ctx->Jq + (long long)(first + k) * ctx->NP * ctx->NP);
      const int rc = copy_instance(ctx, n[k], J[k], stage);
      if (rc) return rc;
      src[k] = stage;
    }
    // padded layout and validation of the whole batch: two launches
    std::vector<LayoutItem> items(count);
    int max_pad = 0;
    for (int k = 0; k < count; ++k) {
      LayoutItem& L = items[k];
      L.src = src[k];
      L.off_mat = (long long)(first + k) * ctx->NP * ctx->NP;
      L.off_vec = (long long)(first + k) * ctx->NP;
      L.n = n[k];
      L.n_pad = pad_of(n[k]);
      L.stats = ctx->stats + (size_t)k * (ctx->NP + 8);
      max_pad = std::max(max_pad, L.n_pad);
    }
    CK(cudaMemsetAsync(ctx->stats, 0, sizeof(double) * (size_t)count * (ctx->NP + 8), ctx->stream));
    CK(cudaMemcpyAsync(ctx->items_d, items.data(), sizeof(LayoutItem) * count, cudaMemcpyHostToDevice, ctx->stream));
    LAUNCH(launch_layout_batch(ctx->P, ctx->items_d, count, max_pad, ctx->J64, ctx->stream));
  } else {
    for (int k = 0; k < count; ++k) {
      int rc = copy_instance(ctx, n[k], J[k], ctx->jstage);
      if (!rc) rc = lay_out_instance(ctx, first + k, k, n[k], ctx->jstage);
      if (rc) return rc;
    }
  }
  const size_t stride = (size_t)ctx->NP + 8;
  std::vector<double> st(stride * count);
  CK(cudaMemcpyAsync(st.data(), ctx->stats, sizeof(double) * st.size(), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  std::vector<InstDesc> ds(count);
  for (int k = 0; k < count; ++k) {
    double sh = 0.0;   // sum_i |h_i| in index order
    for (int i = 0; i < n[k]; ++i) sh += fabs(h[k][i]);
    st[stride * k + 4 + n[k]] = sh;
    const int rc = describe_instance(ctx, first + k, n[k], st.data() + stride * k, ds[k]);
    if (rc) return rc;   // no instance of the batch is added
  }
  const int rc = register_instances(ctx, first, ds);
  if (rc) return rc;
  if (instance_ids)
    for (int k = 0; k < count; ++k) instance_ids[k] = first + k;
  return 0;
}

int qis_clear_instances(qis_ctx* ctx) {
  if (!ctx) return fail(nullptr, QIS_ERR_INVALID_ARG, "ctx is NULL");
  CK(cudaStreamSynchronize(ctx->stream));
  {
    uint64_t c[2];
    int rc = count_candidates(ctx, c);
    if (rc) return rc;
    ctx->cand_acc[0] += c[0];
    ctx->cand_acc[1] += c[1];
    if (ctx->P.B > 0) CK(cudaMemset(ctx->P.nprod, 0, sizeof(int) * (size_t)ctx->P.B));
    if (ctx->P.B > 0) CK(cudaMemset(ctx->P.npair, 0, sizeof(unsigned long long) * (size_t)ctx->P.B));
  }
  CK(cudaMemset(ctx->P.status, 0, sizeof(int)));   // device flags of the removed searches
  ctx->inst.clear();
  ctx->inst_ready.clear();
  ctx->init_pending.clear();
  ctx->init_from_host.clear();
  ctx->e0_valid.clear();
  ctx->e0_deferred.clear();
  ctx->e0_unresolved = false;
  ctx->P.n_inst = 0;
  ctx->P.B = 0;
  ctx->work_dirty = true;
  drop_graph(ctx);
  ctx->merged_fresh = false;
  return 0;
}

int qis_instance_info(qis_ctx* ctx, int instance_id, int* q, int* digits, int* rounded) {
  if (!ctx) return fail(nullptr, QIS_ERR_INVALID_ARG, "ctx is NULL");
  if (instance_id < 0 || instance_id >= (int)ctx->inst.size()) return fail(ctx, QIS_ERR_INVALID_ARG, "bad instance id");
  const InstDesc& d = ctx->inst[instance_id];
  if (q) *q = d.q;
  if (digits) *digits = d.digits;
  if (rounded) *rounded = d.rounded;
  return 0;
}

int qis_instance_n(qis_ctx* ctx, int instance_id, int* n) {
  if (!ctx) return fail(nullptr, QIS_ERR_INVALID_ARG, "ctx is NULL");
  if (instance_id < 0 || instance_id >= (int)ctx->inst.size()) return fail(ctx, QIS_ERR_INVALID_ARG, "bad instance id");
  if (n) *n = ctx->inst[instance_id].n;
  return 0;
}

int qis_init_states(qis_ctx* ctx, int instance_id, const uint64_t* bits) {
  if (!ctx) return fail(nullptr, QIS_ERR_INVALID_ARG, "ctx is NULL");
  if (instance_id < 0 || instance_id >= (int)ctx->inst.size()) return fail(ctx, QIS_ERR_INVALID_ARG, "bad instance id");
  CK(cudaSetDevice(ctx->cfg.device));
  const InstDesc& d = ctx->inst[instance_id];
  const int R = ctx->R, W = d.W, Wm = ctx->Wmax;
  const uint64_t top = (d.n % 64) ? ((1ull << (d.n % 64)) - 1) : ~0ull;
  if (bits)   // checked before anything is written
    for (int r = 0; r < R; ++r)
      if (bits[(size_t)r * W + W - 1] & ~top) return fail(ctx, QIS_ERR_INVALID_ARG, "state bits above n must be zero");
  if (ctx->init_host.size() < (size_t)ctx->max_inst * R * Wm) ctx->init_host.assign((size_t)ctx->max_inst * R * Wm, 0ull);
  uint64_t* h = ctx->init_host.data() + (size_t)d.first_search * Wm;
  std::fill(h, h + (size_t)R * Wm, 0ull);
  if (bits) {
    for (int r = 0; r < R; ++r)
      for (int w = 0; w < W; ++w) h[(size_t)r * Wm + w] = bits[(size_t)r * W + w];
  } else {
    const uint64_t key = state_key(ctx->cfg.seed, instance_id);
    for (int r = 0; r < R; ++r)
      for (int i = 0; i < d.n; ++i)
        if (splitmix64(key, (uint64_t)r * d.n + i) >> 63) h[(size_t)r * Wm + (i >> 6)] |= 1ull << (i & 63);
  }
  // uploaded with the searches' start at the next entry point that needs them (one copy and one
  // launch for every instance set since)
  ctx->init_from_host[instance_id] = 1;
  ctx->init_pending[instance_id] = 1;
  ctx->e0_valid[instance_id] = 0;
  ctx->inst_ready[instance_id] = 1;
  ctx->merged_fresh = false;
  return 0;
}

int qis_init_states_learned(qis_ctx* ctx, int instance_id, qis_mlp* m) {
  if (!ctx) return fail(nullptr, QIS_ERR_INVALID_ARG, "ctx is NULL");
  if (!m) return fail(ctx, QIS_ERR_INVALID_ARG, "network is NULL");
  if (instance_id < 0 || instance_id >= (int)ctx->inst.size()) return fail(ctx, QIS_ERR_INVALID_ARG, "bad instance id");
  const InstDesc& d = ctx->inst[instance_id];
  if (d.n > mlp_max_n(m)) return fail(ctx, QIS_ERR_INVALID_ARG, "instance larger than the network's max_n");
  CK(cudaSetDevice(ctx->cfg.device));
  const uint64_t key = splitmix64(state_key(ctx->cfg.seed, instance_id) ^ 5ull, 0);
  ctx->init_from_host[instance_id] = 0;   // states written on the device replace any pending host ones
  CK(cudaMemsetAsync(ctx->P.init_bits + (size_t)d.first_search * ctx->Wmax, 0,
                     sizeof(uint64_t) * (size_t)ctx->R * ctx->Wmax, ctx->stream));
  CK(mlp_propose_states(m, ctx->J64 + d.off_mat, d.n_pad, ctx->h64 + d.off_vec, d.n, ctx->R, key,
                        ctx->P.init_bits + (size_t)d.first_search * ctx->Wmax, ctx->Wmax, ctx->stream));
  ctx->launches += 5;
  ctx->init_pending[instance_id] = 1;
  ctx->e0_valid[instance_id] = 0;
  ctx->inst_ready[instance_id] = 1;
  ctx->merged_fresh = false;
  CK(cudaStreamSynchronize(ctx->stream));
  return 0;
}

int qis_set_wait_limit(qis_ctx* ctx, uint64_t limit_ns, int probe) {
  if (!ctx) return fail(nullptr, QIS_ERR_INVALID_ARG, "ctx is NULL");
  if (limit_ns < 1000 || limit_ns > 60000000000ull)
    return fail(ctx, QIS_ERR_INVALID_ARG, "limit_ns must be in [1e3, 6e10]");
  if (probe != 0 && probe != 1) return fail(ctx, QIS_ERR_INVALID_ARG, "probe must be 0 or 1");
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->P.wait_ns = limit_ns;
  ctx->P.wait_probe = probe;
  drop_graph(ctx);   // the captured iteration holds the old values
  return 0;
}

int qis_reset(qis_ctx* ctx) {
  if (!ctx) return fail(nullptr, QIS_ERR_INVALID_ARG, "ctx is NULL");
  for (size_t i = 0; i < ctx->inst.size(); ++i)
    if (!ctx->inst_ready[i]) return fail(ctx, QIS_ERR_STATE, "qis_init_states was not called for every instance");
  CK(cudaSetDevice(ctx->cfg.device));
  CK(cudaMemsetAsync(ctx->P.status, 0, sizeof(int), ctx->stream));
  // every search starts again from its stored initial state at the next entry point (one
  // launch; the initial energies as known, or formed by the first iteration of a fused call)
  std::fill(ctx->init_pending.begin(), ctx->init_pending.end(), 1);
  ctx->merged_fresh = false;
  return 0;
}

int qis_iterate(qis_ctx* ctx, int n_iters, int* n_active) {
  if (!ctx) return fail(nullptr, QIS_ERR_INVALID_ARG, "ctx is NULL");
  if (n_iters < 0) return fail(ctx, QIS_ERR_INVALID_ARG, "n_iters must be >= 0");
  {   // searches that start here leave their initial energies to the fused kernel
    const int rc = flush_init(ctx, n_iters > 0 && fused_search(ctx));
    if (rc) return rc;
  }
  if (ctx->inst.empty()) return fail(ctx, QIS_ERR_STATE, "no instance");
  for (size_t i = 0; i < ctx->inst.size(); ++i)
    if (!ctx->inst_ready[i]) return fail(ctx, QIS_ERR_STATE, "qis_init_states was not called for every instance");
  CK(cudaSetDevice(ctx->cfg.device));
  if (ctx->work_dirty) {
    int rc = build_work(ctx);
    if (rc) return rc;
  }
  cudaStream_t s = ctx->stream;
  const DevPtrs& P = ctx->P;
  if (fused_search(ctx) && n_iters > 0) {
    // the kernels of the whole call, captured once per iteration count and replayed
    // a call with the iteration count of the previous one replays a captured graph; the first
    // call with a new count (or after the instances changed) launches directly
    const bool replay = !ctx->profiling && ctx->use_graph && (ctx->graph_n == n_iters || ctx->last_n == n_iters);
    ctx->last_n = n_iters;
    if (replay) {
      if (ctx->graph_exec && ctx->graph_n != n_iters) drop_graph(ctx);
      if (!ctx->graph_exec) {
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        const int rc = launch_iterations_fused(ctx, n_iters, s);
        cudaError_t ec = cudaStreamEndCapture(s, &g);
        if (rc) {
          if (g) cudaGraphDestroy(g);
          return rc;
        }
        CK(ec);
        ec = cudaGraphInstantiate(&ctx->graph_exec, g, 0);
        cudaGraphDestroy(g);
        CK(ec);
        ctx->graph_n = n_iters;
        ctx->launches -= 4;   // counted at each replay below
      }
      CK(cudaGraphLaunch(ctx->graph_exec, s));
      ctx->launches += 4;
    } else {
      const int rc = launch_iterations_fused(ctx, n_iters, s);
      if (rc) return rc;
    }
    ctx->e0_unresolved = false;   // the search kernel that forms the deferred energies is enqueued
  } else if (!ctx->profiling && ctx->use_graph) {
    // one iteration = five kernels, captured once into a CUDA graph and replayed
    if (ctx->graph_exec && ctx->graph_n != 0) drop_graph(ctx);   // a graph of the fused form
    if (!ctx->graph_exec) {
      cudaGraph_t g = nullptr;
      CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      const int rc = launch_iteration(ctx, s);
      cudaError_t ec = cudaStreamEndCapture(s, &g);
      if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
      }
      CK(ec);
      ec = cudaGraphInstantiate(&ctx->graph_exec, g, 0);
      cudaGraphDestroy(g);
      CK(ec);
    }
    for (int it = 0; it < n_iters; ++it) {
      CK(cudaGraphLaunch(ctx->graph_exec, s));
      ctx->launches += ((ctx->cfg.flips == QIS_FLIPS_SINGLE) ? 4 : 5) + (P.inc_on ? 1 : 0);   // kernels in the graph
    }
  } else {
    for (int it = 0; it < n_iters; ++it) {
      const int rc = launch_iteration(ctx, s);
      if (rc) return rc;
    }
  }
  ctx->merged_fresh = false;
  if (n_active) {
    int rc = sync_and_check(ctx);
    if (rc) return rc;
    std::vector<int> act(P.B);
    CK(cudaMemcpy(act.data(), P.active, sizeof(int) * P.B, cudaMemcpyDeviceToHost));
    // a search with every kept state used is inactive from the next pick on; count unused
    std::vector<int> cnt(P.B);
    CK(cudaMemcpy(cnt.data(), P.lst_count, sizeof(int) * P.B, cudaMemcpyDeviceToHost));
    std::vector<uint8_t> used((size_t)P.B * P.K1);
    CK(cudaMemcpy(used.data(), P.lst_used, used.size(), cudaMemcpyDeviceToHost));
    std::vector<int> ord((size_t)P.B * P.K1);
    CK(cudaMemcpy(ord.data(), P.lst_ord, ord.size() * sizeof(int), cudaMemcpyDeviceToHost));
    int na = 0;
    for (int b = 0; b < P.B; ++b) {
      if (!act[b]) continue;
      bool any = false;
      for (int r = 0; r < cnt[b] && !any; ++r) any = !used[(size_t)b * P.K1 + ord[(size_t)b * P.K1 + r]];
      na += any;
    }
    *n_active = na;
  }
  return 0;
}

int qis_search_list(qis_ctx* ctx, int instance_id, int r, uint64_t* bits, double* E, uint8_t* used,
                    uint64_t* stamp, int* count) {
  if (!ctx) return fail(nullptr, QIS_ERR_INVALID_ARG, "ctx is NULL");
  FLUSH_INIT(ctx);
  if (instance_id < 0 || instance_id >= (int)ctx->inst.size()) return fail(ctx, QIS_ERR_INVALID_ARG, "bad instance id");
  if (r < 0 || r >= ctx->R) return fail(ctx, QIS_ERR_INVALID_ARG, "bad search index");
  int rc = sync_and_check(ctx);
  if (rc) return rc;
  const InstDesc& d = ctx->inst[instance_id];
  const int K1 = ctx->K1, Wm = ctx->Wmax;
  const size_t b = (size_t)d.first_search + r;
  int cnt = 0;
  CK(cudaMemcpy(&cnt, ctx->P.lst_count + b, sizeof(int), cudaMemcpyDeviceToHost));
  std::vector<int> ord(K1);
  std::vector<double> e(K1);
  std::vector<uint64_t> st(K1), bb((size_t)K1 * Wm);
  std::vector<uint8_t> u(K1);
  CK(cudaMemcpy(ord.data(), ctx->P.lst_ord + b * K1, K1 * sizeof(int), cudaMemcpyDeviceToHost));
  if (ctx->mode == QIS_FP64) {
    CK(cudaMemcpy(e.data(), ctx->P.lst_E + b * K1, K1 * sizeof(double), cudaMemcpyDeviceToHost));
  } else {   // the exact integer E 2^q, scaled by 2^-q as on the device
    std::vector<long long> q(K1);
    CK(cudaMemcpy(q.data(), ctx->P.lst_q + b * K1, K1 * sizeof(long long), cudaMemcpyDeviceToHost));
    for (int k = 0; k < K1; ++k) e[k] = ldexp((double)q[k], -d.q);
  }
  CK(cudaMemcpy(st.data(), ctx->P.lst_stamp + b * K1, K1 * sizeof(uint64_t), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(u.data(), ctx->P.lst_used + b * K1, K1, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(bb.data(), ctx->P.lst_bits + b * K1 * Wm, bb.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost));
  for (int k = 0; k < cnt; ++k) {
    const int slot = ord[k];
    if (bits) memcpy(bits + (size_t)k * d.W, &bb[(size_t)slot * Wm], d.W * sizeof(uint64_t));
    if (E) E[k] = e[slot];
    if (used) used[k] = u[slot];
    if (stamp) stamp[k] = st[slot];
  }
  if (count) *count = cnt;
  return 0;
}

namespace {

// Write one search's kept list (entries in key order) into the device list of search b. The
// caller has validated the arguments; hashes are computed on the device from the bits.
int flush_init(qis_ctx* ctx, bool defer);

int import_search(qis_ctx* ctx, int b, int W, int q, int count, const uint64_t* bits, const double* E,
                  const uint8_t* used, const uint64_t* stamp, int t) {
  {   // a pending start of the instance's searches comes first (its initial energies stay)
    const int rc = flush_init(ctx, false);
    if (rc) return rc;
  }
  const int K1 = ctx->K1, Wm = ctx->Wmax;
  const size_t base = (size_t)b * K1;
  std::vector<uint64_t> lb((size_t)K1 * Wm, 0ull), st(K1, 0ull);
  std::vector<double> e(K1, INFINITY);
  std::vector<long long> eq(K1, 0);
  std::vector<unsigned long long> key(K1, ~0ull);
  std::vector<uint8_t> u(K1, 0);
  std::vector<int> ord(K1, -1);
  int act = 0;
  for (int k = 0; k < count; ++k) {
    memcpy(&lb[(size_t)k * Wm], bits + (size_t)k * W, W * sizeof(uint64_t));
    e[k] = E[k];
    eq[k] = (ctx->mode != QIS_FP64) ? llrint(ldexp(E[k], q)) : 0;   // exact on the grid
    if (ctx->mode != QIS_FP64) {
      key[k] = qkey(eq[k]);
    } else {   // order key of a double (as dkey on the device)
      uint64_t u;
      const double x = E[k] + 0.0;
      memcpy(&u, &x, 8);
      key[k] = (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
    }
    u[k] = used ? (used[k] != 0) : 0;
    st[k] = stamp ? stamp[k] : (uint64_t)k;
    ord[k] = k;
    act |= !u[k];
  }
  // fields by update need the generating parent's ring entry: none for imported entries
  int t0 = t;
  for (int k = 0; k < count; ++k) t0 = std::max(t0, (int)std::min<uint64_t>(st[k] >> 32, 0x7fffffff));
  const int one[5] = {count, act, t, 0, t0};
  cudaStream_t s = ctx->stream;
  const DevPtrs& P = ctx->P;
  CK(cudaMemcpyAsync(P.lst_bits + base * Wm, lb.data(), lb.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(P.lst_E + base, e.data(), K1 * sizeof(double), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(P.lst_q + base, eq.data(), K1 * sizeof(long long), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(P.lst_key + base, key.data(), K1 * sizeof(unsigned long long), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(P.lst_stamp + base, st.data(), K1 * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(P.lst_used + base, u.data(), K1, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(P.lst_ord + base, ord.data(), K1 * sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(P.lst_count + b, &one[0], sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(P.active + b, &one[1], sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(P.iter_t + b, &one[2], sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(P.surv_cnt + b, &one[3], sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(P.ring_t0 + b, &one[4], sizeof(int), cudaMemcpyHostToDevice, s));
  LAUNCH(launch_hash_list(P, b, count, s));
  CK(cudaStreamSynchronize(s));   // the host vectors above are the copies' sources
  return 0;
}

// Checks of an imported list: 1 <= count <= K+1, no bits above n, finite nondecreasing E,
// distinct states.
int check_list(qis_ctx* ctx, int n, int count, const uint64_t* bits, const double* E) {
  const int W = words_of(n);
  if (count < 1 || count > ctx->K1) return fail(ctx, QIS_ERR_INVALID_ARG, "list length must be in [1, K+1]");
  if (!bits || !E) return fail(ctx, QIS_ERR_INVALID_ARG, "bits and E must not be NULL");
  const uint64_t top = (n % 64) ? ((1ull << (n % 64)) - 1) : ~0ull;
  std::vector<std::vector<uint64_t>> v;
  for (int k = 0; k < count; ++k) {
    if (bits[(size_t)k * W + W - 1] & ~top) return fail(ctx, QIS_ERR_INVALID_ARG, "state bits above n must be zero");
    if (!std::isfinite(E[k])) return fail(ctx, QIS_ERR_INVALID_ARG, "list energies must be finite");
    if (k > 0 && E[k] < E[k - 1]) return fail(ctx, QIS_ERR_INVALID_ARG, "list energies must be nondecreasing");
    v.emplace_back(bits + (size_t)k * W, bits + (size_t)(k + 1) * W);
  }
  std::sort(v.begin(), v.end());
  if (std::adjacent_find(v.begin(), v.end()) != v.end())
    return fail(ctx, QIS_ERR_INVALID_ARG, "list states must be distinct");
  return 0;
}

}  // namespace

int qis_set_search_list(qis_ctx* ctx, int instance_id, int r, int count, const uint64_t* bits, const double* E,
                        const uint8_t* used, const uint64_t* stamp, int t) {
  if (!ctx) return fail(nullptr, QIS_ERR_INVALID_ARG, "ctx is NULL");
  FLUSH_INIT(ctx);
  if (instance_id < 0 || instance_id >= (int)ctx->inst.size()) return fail(ctx, QIS_ERR_INVALID_ARG, "bad instance id");
  if (r < 0 || r >= ctx->R) return fail(ctx, QIS_ERR_INVALID_ARG, "bad search index");
  if (t < 0) return fail(ctx, QIS_ERR_INVALID_ARG, "iteration counter must be >= 0");
  const InstDesc& d = ctx->inst[instance_id];
  int rc = check_list(ctx, d.n, count, bits, E);
  if (rc) return rc;
  CK(cudaSetDevice(ctx->cfg.device));
  rc = sync_and_check(ctx);
  if (rc) return rc;
  rc = import_search(ctx, d.first_search + r, d.W, d.q, count, bits, E, used, stamp, t);
  if (rc) return rc;
  ctx->merged_fresh = false;
  return 0;
}

// ---------------------------------------------------------------- checkpoint / resume
// File layout (little endian): "QISCKPT1", int32 {version, K, R, precision, n_instances, flips},
// uint64 seed; per instance: int32 {n, ready}, J (n*n FP64 row major), h (n FP64), the R
// initial states (R*W uint64); per search of the instance: int32 {count, t, active, 0}, then
// count entries {W uint64 bits, FP64 E, uint64 stamp, uint64 used}; last, the FNV-1a 64-bit
// hash of every byte before it.
namespace {

constexpr char kCkptMagic[8] = {'Q', 'I', 'S', 'C', 'K', 'P', 'T', '1'};
constexpr int kCkptVersion = 1;

struct Fnv1a {
  uint64_t h = 0xcbf29ce484222325ull;
  void add(const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
      h ^= c[i];
      h *= 0x100000001b3ull;
    }
  }
};

struct Writer {
  FILE* f;
  Fnv1a sum;
  bool ok = true;
  void put(const void* p, size_t n) {
    if (n == 0) return;
    ok = ok && fwrite(p, 1, n, f) == n;
    sum.add(p, n);
  }
};

struct Reader {
  std::vector<unsigned char> data;
  size_t pos = 0;
  bool get(void* p, size_t n) {
    if (pos + n > data.size()) return false;
    memcpy(p, data.data() + pos, n);
    pos += n;
    return true;
  }
};

}  // namespace

int qis_save(qis_ctx* ctx, const char* path) {
  if (!ctx) return fail(nullptr, QIS_ERR_INVALID_ARG, "ctx is NULL");
  FLUSH_INIT(ctx);
  if (!path) return fail(ctx, QIS_ERR_INVALID_ARG, "path is NULL");
  CK(cudaSetDevice(ctx->cfg.device));
  int rc = sync_and_check(ctx);
  if (rc) return rc;
  FILE* f = fopen(path, "wb");
  if (!f) return fail(ctx, QIS_ERR_INVALID_ARG, std::string("cannot open ") + path + " for writing");
  Writer w{f};
  const int K1 = ctx->K1, Wm = ctx->Wmax, R = ctx->R;
  const int hdr[6] = {kCkptVersion, ctx->cfg.K, R, ctx->mode, (int)ctx->inst.size(), ctx->cfg.flips};
  w.put(kCkptMagic, 8);
  w.put(hdr, sizeof(hdr));
  w.put(&ctx->cfg.seed, 8);
  auto bail = [&](int code) {   // the message is already in ctx->err
    fclose(f);
    remove(path);
    return code;
  };
  for (size_t id = 0; id < ctx->inst.size(); ++id) {
    const InstDesc& d = ctx->inst[id];
    const int n = d.n, W = d.W;
    const int ih[2] = {n, ctx->inst_ready[id]};
    w.put(ih, sizeof(ih));
    std::vector<double> J((size_t)n * n), h(n);
    cudaError_t e = cudaMemcpy2D(J.data(), sizeof(double) * n, ctx->J64 + d.off_mat, sizeof(double) * d.n_pad,
                                 sizeof(double) * n, n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(h.data(), ctx->h64 + d.off_vec, sizeof(double) * n, cudaMemcpyDeviceToHost);
    std::vector<uint64_t> ib((size_t)R * Wm);
    if (e == cudaSuccess)
      e = cudaMemcpy(ib.data(), ctx->P.init_bits + (size_t)d.first_search * Wm, ib.size() * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return bail(fail(ctx, QIS_ERR_CUDA, std::string("checkpoint copy: ") + cudaGetErrorString(e)));
    }
    w.put(J.data(), J.size() * 8);
    w.put(h.data(), h.size() * 8);
    for (int r = 0; r < R; ++r) w.put(&ib[(size_t)r * Wm], W * 8);
    std::vector<uint64_t> bits((size_t)K1 * W), stamp(K1);
    std::vector<double> E(K1);
    std::vector<uint8_t> used(K1);
    for (int r = 0; r < R; ++r) {
      const int b = d.first_search + r;
      int cnt = 0, t = 0, act = 0;
      rc = qis_search_list(ctx, (int)id, r, bits.data(), E.data(), used.data(), stamp.data(), &cnt);
      if (rc) return bail(rc);
      e = cudaMemcpy(&t, ctx->P.iter_t + b, sizeof(int), cudaMemcpyDeviceToHost);
      if (e == cudaSuccess) e = cudaMemcpy(&act, ctx->P.active + b, sizeof(int), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(ctx, QIS_ERR_CUDA, std::string("checkpoint copy: ") + cudaGetErrorString(e)));
      }
      const int sh[4] = {cnt, t, act, 0};
      w.put(sh, sizeof(sh));
      for (int k = 0; k < cnt; ++k) {
        const uint64_t u = used[k];
        w.put(&bits[(size_t)k * W], W * 8);
        w.put(&E[k], 8);
        w.put(&stamp[k], 8);
        w.put(&u, 8);
      }
    }
  }
  const uint64_t sum = w.sum.h;
  w.put(&sum, 8);
  const bool ok = w.ok && fclose(f) == 0;
  if (!ok) {
    remove(path);
    return fail(ctx, QIS_ERR_INVALID_ARG, std::string("write to ") + path + " failed");
  }
  return 0;
}

namespace {
int load_checkpoint(qis_ctx* ctx, const char* path);
}

int qis_load(qis_ctx* ctx, const char* path) {
  if (!ctx) return fail(nullptr, QIS_ERR_INVALID_ARG, "ctx is NULL");
  if (!path) return fail(ctx, QIS_ERR_INVALID_ARG, "path is NULL");
  if (!ctx->inst.empty()) return fail(ctx, QIS_ERR_STATE, "qis_load needs a context without instances");
  const int rc = load_checkpoint(ctx, path);
  if (rc && !ctx->inst.empty()) {
    // a file that fails part-way leaves no partly restored context: the instances created
    // before the failing record are removed, so the caller can retry with another file
    const std::string msg = ctx->err;
    qis_clear_instances(ctx);
    ctx->err = msg;
  }
  return rc;
}

namespace {
int load_checkpoint(qis_ctx* ctx, const char* path) {
  Reader rd;
  {
    FILE* f = fopen(path, "rb");
    if (!f) return fail(ctx, QIS_ERR_INVALID_ARG, std::string("cannot open ") + path);
    unsigned char buf[1 << 16];
    size_t got;
    while ((got = fread(buf, 1, sizeof(buf), f)) > 0) rd.data.insert(rd.data.end(), buf, buf + got);
    fclose(f);
  }
  const auto corrupt = [&](const char* what) {
    return fail(ctx, QIS_ERR_INVALID_ARG, std::string("checkpoint ") + path + ": " + what);
  };
  if (rd.data.size() < 8 + 24 + 8 + 8) return corrupt("file too short");
  {
    Fnv1a s;
    s.add(rd.data.data(), rd.data.size() - 8);
    uint64_t stored;
    memcpy(&stored, rd.data.data() + rd.data.size() - 8, 8);
    if (s.h != stored) return corrupt("checksum mismatch");
  }
  char magic[8];
  int hdr[6];
  uint64_t seed;
  rd.get(magic, 8);
  rd.get(hdr, sizeof(hdr));
  rd.get(&seed, 8);
  if (memcmp(magic, kCkptMagic, 8) != 0) return corrupt("not a checkpoint");
  if (hdr[0] != kCkptVersion) return corrupt("unsupported version");
  if (hdr[1] != ctx->cfg.K || hdr[2] != ctx->R || hdr[3] != ctx->mode || hdr[5] != ctx->cfg.flips)
    return fail(ctx, QIS_ERR_INVALID_ARG, "checkpoint K, R, precision or flip set differ from the context's");
  const int n_inst = hdr[4], R = ctx->R;
  if (n_inst < 0 || n_inst > ctx->max_inst) return fail(ctx, QIS_ERR_INVALID_ARG, "checkpoint has too many instances");
  const size_t end = rd.data.size() - 8;
  for (int id = 0; id < n_inst; ++id) {
    int ih[2];
    if (!rd.get(ih, sizeof(ih))) return corrupt("truncated");
    const int n = ih[0];
    if (n < 2 || n > ctx->cfg.max_n) return fail(ctx, QIS_ERR_INVALID_ARG, "checkpoint instance larger than max_n");
    const int W = words_of(n);
    std::vector<double> J((size_t)n * n), h(n);
    if (!rd.get(J.data(), J.size() * 8) || !rd.get(h.data(), h.size() * 8)) return corrupt("truncated");
    std::vector<uint64_t> ib((size_t)R * W);
    if (!rd.get(ib.data(), ib.size() * 8)) return corrupt("truncated");
    int got = -1;
    int rc = qis_create_instance(ctx, n, J.data(), h.data(), &got);
    if (rc) return rc;
    const InstDesc& d = ctx->inst[got];
    if (ih[1]) {
      rc = qis_init_states(ctx, got, ib.data());
      if (rc) return rc;
    }
    for (int r = 0; r < R; ++r) {
      int sh[4];
      if (!rd.get(sh, sizeof(sh))) return corrupt("truncated");
      const int cnt = sh[0];
      if (cnt < 0 || cnt > ctx->K1) return corrupt("bad list length");
      std::vector<uint64_t> bits((size_t)cnt * W), stamp(cnt);
      std::vector<double> E(cnt);
      std::vector<uint8_t> used(cnt);
      for (int k = 0; k < cnt; ++k) {
        uint64_t u;
        if (!rd.get(&bits[(size_t)k * W], W * 8) || !rd.get(&E[k], 8) || !rd.get(&stamp[k], 8) || !rd.get(&u, 8))
          return corrupt("truncated");
        used[k] = (uint8_t)(u != 0);
      }
      if (!ih[1]) continue;   // lists of an instance without initial states are not restored
      rc = check_list(ctx, n, cnt, bits.data(), E.data());
      if (rc) return rc;
      rc = import_search(ctx, d.first_search + r, W, d.q, cnt, bits.data(), E.data(), used.data(), stamp.data(), sh[1]);
      if (rc) return rc;
      const int act = sh[2];
      CK(cudaMemcpy(ctx->P.active + d.first_search + r, &act, sizeof(int), cudaMemcpyHostToDevice));
    }
  }
  if (rd.pos != end) return corrupt("trailing bytes");
  ctx->merged_fresh = false;
  return 0;
}
}  // namespace

int qis_topk_states(qis_ctx* ctx, int instance_id, int k, uint64_t* bits_out, double* E_out, uint64_t* src_out,
                    int* n_out) {
  if (!ctx) return fail(nullptr, QIS_ERR_INVALID_ARG, "ctx is NULL");
  FLUSH_INIT(ctx);
  if (instance_id < 0 || instance_id >= (int)ctx->inst.size()) return fail(ctx, QIS_ERR_INVALID_ARG, "bad instance id");
  if (k < 0) return fail(ctx, QIS_ERR_INVALID_ARG, "k must be >= 0");
  CK(cudaSetDevice(ctx->cfg.device));
  cudaStream_t s = ctx->stream;
  if (!ctx->merged_fresh) {
    LAUNCH(launch_final_merge(ctx->P, s));
    ctx->merged_fresh = true;
    ctx->counts_valid = false;
  }
  if (!ctx->counts_valid) {   // once per merge: the status check and every instance's count
    int rc = sync_and_check(ctx);
    if (rc) return rc;
    ctx->mrg_counts.assign(ctx->inst.size(), 0);
    CK(cudaMemcpy(ctx->mrg_counts.data(), ctx->P.mrg_count, sizeof(int) * ctx->inst.size(), cudaMemcpyDeviceToHost));
    ctx->counts_valid = true;
  }
  const InstDesc& d = ctx->inst[instance_id];
  const int cnt = ctx->mrg_counts[instance_id];
  const int m = k < cnt ? k : cnt;
  for (int off = 0; off < m; off += ctx->scratch_states) {
    const int c = (m - off < ctx->scratch_states) ? m - off : ctx->scratch_states;
    // gather rows off..off+c of the merged list
    DevPtrs Q = ctx->P;
    Q.mrg_ref = ctx->P.mrg_ref + off;   // shift the view so row 0 is entry `off`
    LAUNCH(launch_gather_merged(Q, instance_id, d, c, ctx->scratch_bits, s));
    LAUNCH(launch_rescore(ctx->P, d, ctx->scratch_bits, c, d.W, ctx->scratch_E, s));
    if (bits_out) CK(cudaMemcpyAsync(bits_out + (size_t)off * d.W, ctx->scratch_bits, sizeof(uint64_t) * c * d.W,
                                     cudaMemcpyDeviceToHost, s));
    if (E_out) CK(cudaMemcpyAsync(E_out + off, ctx->scratch_E, sizeof(double) * c, cudaMemcpyDeviceToHost, s));
    if (src_out && off == 0)
      CK(cudaMemcpyAsync(src_out, ctx->P.mrg_src + (size_t)instance_id * ctx->K1, sizeof(uint64_t) * m,
                         cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  if (n_out) *n_out = m;
  return 0;
}

int qis_topk_states_all(qis_ctx* ctx, int k, uint64_t* bits_out, double* E_out, uint64_t* src_out, int* n_out) {
  if (!ctx) return fail(nullptr, QIS_ERR_INVALID_ARG, "ctx is NULL");
  FLUSH_INIT(ctx);
  if (k < 0 || k > ctx->K1) return fail(ctx, QIS_ERR_INVALID_ARG, "k must be in [0, K+1]");
  if (ctx->inst.empty()) return fail(ctx, QIS_ERR_STATE, "no instance");
  CK(cudaSetDevice(ctx->cfg.device));
  cudaStream_t s = ctx->stream;
  if (!ctx->merged_fresh) {
    LAUNCH(launch_final_merge(ctx->P, s));
    ctx->merged_fresh = true;
    ctx->counts_valid = false;
  }
  const int ni = (int)ctx->inst.size(), Wm = ctx->Wmax;
  if (k > 0) {
    bool exact = ctx->mode != QIS_FP64;
    int max_n = 0;
    for (const InstDesc& d : ctx->inst) {
      exact = exact && !d.rounded;
      max_n = std::max(max_n, d.n);
    }
    LAUNCH(launch_topk_all(ctx->P, k, exact, max_n, ctx->all_bits, ctx->all_E, s));
  }
  int rc = sync_and_check(ctx);
  if (rc) return rc;
  ctx->mrg_counts.assign(ni, 0);
  CK(cudaMemcpy(ctx->mrg_counts.data(), ctx->P.mrg_count, sizeof(int) * ni, cudaMemcpyDeviceToHost));
  ctx->counts_valid = true;
  if (k > 0) {
    if (bits_out) CK(cudaMemcpyAsync(bits_out, ctx->all_bits, sizeof(uint64_t) * (size_t)ni * k * Wm, cudaMemcpyDeviceToHost, s));
    if (E_out) CK(cudaMemcpyAsync(E_out, ctx->all_E, sizeof(double) * (size_t)ni * k, cudaMemcpyDeviceToHost, s));
    if (src_out) CK(cudaMemcpy2DAsync(src_out, sizeof(uint64_t) * k, ctx->P.mrg_src, sizeof(uint64_t) * ctx->K1,
                                      sizeof(uint64_t) * k, ni, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  if (n_out)
    for (int i = 0; i < ni; ++i) n_out[i] = std::min(k, ctx->mrg_counts[i]);
  return 0;
}

int qis_merge(qis_ctx* ctx) {
  if (!ctx) return fail(nullptr, QIS_ERR_INVALID_ARG, "ctx is NULL");
  FLUSH_INIT(ctx);
  if (ctx->inst.empty()) return fail(ctx, QIS_ERR_STATE, "no instance");
  CK(cudaSetDevice(ctx->cfg.device));
  LAUNCH(launch_final_merge(ctx->P, ctx->stream));
  ctx->merged_fresh = true;
  ctx->counts_valid = false;
  return 0;
}

int qis_energies(qis_ctx* ctx, int instance_id, int count, const uint64_t* bits, double* E_out) {
  if (!ctx) return fail(nullptr, QIS_ERR_INVALID_ARG, "ctx is NULL");
  if (instance_id < 0 || instance_id >= (int)ctx->inst.size()) return fail(ctx, QIS_ERR_INVALID_ARG, "bad instance id");
  if (count < 0 || (count > 0 && (!bits || !E_out))) return fail(ctx, QIS_ERR_INVALID_ARG, "bad buffers");
  CK(cudaSetDevice(ctx->cfg.device));
  const InstDesc& d = ctx->inst[instance_id];
  cudaStream_t s = ctx->stream;
  for (int off = 0; off < count; off += ctx->scratch_states) {
    const int c = (count - off < ctx->scratch_states) ? count - off : ctx->scratch_states;
    CK(cudaMemcpyAsync(ctx->scratch_bits, bits + (size_t)off * d.W, sizeof(uint64_t) * c * d.W, cudaMemcpyHostToDevice, s));
    LAUNCH(launch_rescore(ctx->P, d, ctx->scratch_bits, c, d.W, ctx->scratch_E, s));
    CK(cudaMemcpyAsync(E_out + off, ctx->scratch_E, sizeof(double) * c, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  return 0;
}

int qis_synchronize(qis_ctx* ctx) {
  if (!ctx) return fail(nullptr, QIS_ERR_INVALID_ARG, "ctx is NULL");
  FLUSH_INIT(ctx);
  return sync_and_check(ctx);
}

int qis_kernel_launches(qis_ctx* ctx, uint64_t* count) {
  if (!ctx || !count) return fail(ctx, QIS_ERR_INVALID_ARG, "NULL argument");
  *count = ctx->launches;
  return 0;
}


int qis_candidate_count(qis_ctx* ctx, uint64_t* pairs, uint64_t* singles) {
  if (!ctx) return fail(nullptr, QIS_ERR_INVALID_ARG, "ctx is NULL");
  FLUSH_INIT(ctx);
  CK(cudaStreamSynchronize(ctx->stream));
  uint64_t c[2];
  int rc = count_candidates(ctx, c);
  if (rc) return rc;
  if (pairs) *pairs = ctx->cand_acc[0] + c[0];
  if (singles) *singles = ctx->cand_acc[1] + c[1];
  return 0;
}

int qis_survivor_count(qis_ctx* ctx, uint64_t* count) {
  if (!ctx || !count) return fail(ctx, QIS_ERR_INVALID_ARG, "NULL argument");
  FLUSH_INIT(ctx);
  CK(cudaStreamSynchronize(ctx->stream));
  unsigned long long v[64];
  CK(cudaMemcpy(v, ctx->P.surv_tot, sizeof(v), cudaMemcpyDeviceToHost));
  uint64_t t = 0;
  for (int k = 0; k < 64; ++k) t += v[k];
  *count = t;
  return 0;
}

int qis_evaluated_pairs(qis_ctx* ctx, uint64_t* pairs) {
  if (!ctx || !pairs) return fail(ctx, QIS_ERR_INVALID_ARG, "NULL argument");
  FLUSH_INIT(ctx);
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->mode == QIS_FP64) {   // the plain form evaluates every pair
    uint64_t c[2];
    int rc = count_candidates(ctx, c);
    if (rc) return rc;
    *pairs = ctx->cand_acc[0] + c[0];
    return 0;
  }
  unsigned long long v[64];
  CK(cudaMemcpy(v, ctx->P.eval_cnt, sizeof(v), cudaMemcpyDeviceToHost));
  uint64_t t = 0;
  for (int k = 0; k < 64; ++k) t += v[k];
  *pairs = t;
  return 0;
}

int qis_get_tuning(qis_ctx* ctx, qis_tuning* out) {
  if (!ctx || !out) return fail(ctx, QIS_ERR_INVALID_ARG, "NULL argument");
  *out = ctx->tune;
  out->pair_scan = sparse_scan(ctx) ? 1 : 2;
  if (out->scan_search_group == 0) out->scan_search_group = ctx->R;
  if (out->gemm_tile_searches == 0) out->gemm_tile_searches = gemm_tile_n(ctx->R, ctx->digits_used);
  return 0;
}

int qis_set_incremental_fields(qis_ctx* ctx, int on) {
  if (!ctx) return fail(nullptr, QIS_ERR_INVALID_ARG, "ctx is NULL");
  if (on != 0 && on != 1) return fail(ctx, QIS_ERR_INVALID_ARG, "on must be 0 or 1");
  if (on && (ctx->mode == QIS_FP64 || ctx->fields_simt))
    return fail(ctx, QIS_ERR_INVALID_ARG, "fields by update need the split modes and the tensor-core field GEMM");
  if (ctx->P.inc_on != on) {
    ctx->P.inc_on = on;
    drop_graph(ctx);   // the iteration's kernel sequence changes
  }
  return 0;
}

int qis_set_tuning(qis_ctx* ctx, const qis_tuning* t) {
  if (!ctx || !t) return fail(ctx, QIS_ERR_INVALID_ARG, "NULL argument");
  if (t->scan_chunk_nc < 1 || t->scan_chunk_nc > 8) return fail(ctx, QIS_ERR_INVALID_ARG, "scan_chunk_nc must be in [1, 8]");
  if (t->scan_search_group < 0 || t->scan_search_group > ctx->R)
    return fail(ctx, QIS_ERR_INVALID_ARG, "scan_search_group must be in [0, R]");
  const int nt = t->gemm_tile_searches;
  if (nt != 0 && (nt % 16 != 0 || nt < 16 || nt > 256 || ctx->digits_used * nt > 512))
    return fail(ctx, QIS_ERR_INVALID_ARG, "gemm_tile_searches must be a multiple of 16 in [16, 256] with digits * it <= 512");
  if (t->pair_scan < 0 || t->pair_scan > 3) return fail(ctx, QIS_ERR_INVALID_ARG, "pair_scan must be 0, 1, 2 or 3");
  if ((t->pair_scan == 1 || t->pair_scan == 3) && !sparse_allowed(ctx))
    return fail(ctx, QIS_ERR_INVALID_ARG, "the output-sensitive scan needs a split mode and a padded size <= 4096");
  CK(cudaSetDevice(ctx->cfg.device));
  CK(cudaStreamSynchronize(ctx->stream));
  const qis_tuning old = ctx->tune;
  ctx->tune = *t;
  ctx->work_dirty = true;
  drop_graph(ctx);
  if (!ctx->inst.empty()) {
    const int rc = build_work(ctx);
    if (rc) {
      ctx->tune = old;
      ctx->work_dirty = true;
      return rc;
    }
  }
  return 0;
}

int qis_autotune(qis_ctx* ctx, int iters, qis_tuning* best, double* best_ms) {
  if (!ctx) return fail(nullptr, QIS_ERR_INVALID_ARG, "ctx is NULL");
  FLUSH_INIT(ctx);
  if (iters < 1) return fail(ctx, QIS_ERR_INVALID_ARG, "iters must be >= 1");
  if (ctx->inst.empty()) return fail(ctx, QIS_ERR_STATE, "no instance");
  for (size_t i = 0; i < ctx->inst.size(); ++i)
    if (!ctx->inst_ready[i]) return fail(ctx, QIS_ERR_STATE, "qis_init_states was not called for every instance");
  CK(cudaSetDevice(ctx->cfg.device));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  // time of `iters` iterations from the initial states (the first replay builds the graph, so
  // every candidate runs once untimed)
  auto trial = [&](const qis_tuning& t, double* ms) -> int {
    int rc = qis_set_tuning(ctx, &t);
    if (rc) return rc;
    for (int rep = 0; rep < 2; ++rep) {
      rc = qis_reset(ctx);
      if (rc) return rc;
      CK(cudaEventRecord(e0, ctx->stream));
      rc = qis_iterate(ctx, iters, nullptr);
      if (rc) return rc;
      CK(cudaEventRecord(e1, ctx->stream));
      rc = sync_and_check(ctx);
      if (rc) return rc;
    }
    float f = 0.f;
    CK(cudaEventElapsedTime(&f, e0, e1));
    *ms = f;
    return 0;
  };
  qis_tuning cur = ctx->tune;
  cur.scan_search_group = cur.scan_search_group ? cur.scan_search_group : ctx->R;
  double cur_ms = 0.0;
  int rc = trial(cur, &cur_ms);
  // a candidate the instance set cannot take (QIS_ERR_INVALID_ARG) is skipped; any other
  // failure ends the search
  auto consider = [&](const qis_tuning& t) {
    if (rc) return;
    double ms = 0.0;
    const int r = trial(t, &ms);
    if (r == 0 && ms < cur_ms) {
      cur = t;
      cur_ms = ms;
    } else if (r != 0 && r != QIS_ERR_INVALID_ARG) {
      rc = r;
    }
  };
  // coordinate search: scan form, then chunk width and search group (the dense form's
  // shapes), GEMM tile, each with the others fixed
  cur.pair_scan = sparse_scan(ctx) ? 1 : 2;
  if (sparse_allowed(ctx)) {
    qis_tuning t = cur;
    t.pair_scan = 3 - cur.pair_scan;
    consider(t);
  }
  for (int nc : {8, 6, 4, 2}) {
    if (cur.pair_scan == 1) break;
    qis_tuning t = cur;
    t.scan_chunk_nc = nc;
    if (nc != cur.scan_chunk_nc) consider(t);
  }
  for (int div = 2; div <= 16 && cur.pair_scan != 1; div *= 2) {
    qis_tuning t = cur;
    t.scan_search_group = (ctx->R + div - 1) / div;
    if (t.scan_search_group >= 4 && t.scan_search_group != cur.scan_search_group) consider(t);
  }
  if (ctx->mode != QIS_FP64) {
    for (int nt = 16; nt <= 256; nt *= 2) {
      if (ctx->digits_used * nt > 512 || nt > ((ctx->R + 15) / 16) * 16) continue;
      qis_tuning t = cur;
      t.gemm_tile_searches = nt;
      if (nt != cur.gemm_tile_searches) consider(t);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  rc = qis_set_tuning(ctx, &cur);
  if (rc) return rc;
  rc = qis_reset(ctx);
  if (rc) return rc;
  if (best) *best = cur;
  if (best_ms) *best_ms = cur_ms;
  return 0;
}

int qis_get_stream(qis_ctx* ctx, void** stream) {
  if (!ctx || !stream) return fail(ctx, QIS_ERR_INVALID_ARG, "NULL argument");
  *stream = (void*)ctx->stream;
  return 0;
}

int qis_profile_enable(qis_ctx* ctx, int on) {
  if (!ctx) return fail(nullptr, QIS_ERR_INVALID_ARG, "ctx is NULL");
  ctx->profiling = on != 0;
  return 0;
}

int qis_profile_query(qis_ctx* ctx, int kernel_class, double* total_ms, uint64_t* launches) {
  if (!ctx) return fail(nullptr, QIS_ERR_INVALID_ARG, "ctx is NULL");
  if (kernel_class < 0 || kernel_class >= 6) return fail(ctx, QIS_ERR_INVALID_ARG, "kernel class must be in [0, 6)");
  CK(cudaStreamSynchronize(ctx->stream));
  double sum = 0.0;
  auto& v = ctx->ev[kernel_class];
  for (size_t k = 0; k < ctx->ev_used[kernel_class]; ++k) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, v[k].first, v[k].second));
    sum += ms;
  }
  if (total_ms) *total_ms = sum;
  if (launches) *launches = ctx->ev_used[kernel_class];
  ctx->ev_used[kernel_class] = 0;
  return 0;
}

}  // extern "C"
