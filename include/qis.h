/*
 * qis.h -- C ABI of the GB300 quantum-inspired (QI) search library (libqis.so).
 *
 * The method is the QI search of Ueda, Otsuka and Yunoki (arXiv 2010.00180) for
 * low-energy states of the classical Ising Hamiltonian
 *     H0 = sum_{i<j} J_ij s_i s_j + sum_i h_i s_i                          (Eq. (1))
 * Each search keeps K+1 product states sorted by energy (Alg. 2); every iteration takes
 * the first unused kept state as the parent, generates all its single flips X_i and
 * pair flips X_i X_j (the flip sets of Sec. III, H1 of Eq. (H1)), and keeps the K+1
 * lowest distinct states (Alg. 3). R independent searches per instance start from R
 * initial states and their lists are merged at the end (Alg. 4, R = L).
 *
 * Conventions shared by every entry point:
 *  - States are packed bits, W = ceil(n/64) little-endian uint64 words per state; bit i
 *    is sigma_i of Eq. (4) and sigma_i = 1 means s_i = -1. Bits above n must be zero.
 *  - Every pointer in this header is a HOST pointer. The caller owns all buffers; the
 *    library copies what it needs before returning and never keeps a caller pointer.
 *  - Return value: 0 on success, a negative QIS_ERR_* code on failure. The failing
 *    call leaves a message for qis_last_error(). A context is used by one host thread
 *    at a time.
 *  - Kept lists are ordered by the key (E, stamp): ascending energy, ties broken by
 *    arrival, which is the order Alg. 2 produces by inserting a new state after every
 *    kept state of equal energy. stamp = 0 for the initial state and (t << 32) | c for
 *    candidate c (c = i for the single flip of site i, c = n + rank(i, j) for the pair
 *    i < j in lexicographic order) generated in iteration t (1-based).
 *  - Device work runs on the library's own CUDA stream. qis_iterate and qis_reset are
 *    asynchronous; calls that return data to the host synchronise that stream.
 */
#ifndef QIS_H
#define QIS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes. */
#define QIS_OK 0
#define QIS_ERR_INVALID_ARG (-1)  /* bad size, K, pointer, non-symmetric J, nonzero diagonal, NaN/Inf, ... */
#define QIS_ERR_OOM (-2)          /* device allocation failed */
#define QIS_ERR_CUDA (-3)         /* a CUDA runtime call failed */
#define QIS_ERR_DEVICE_TIMEOUT (-4) /* a bounded device-side wait gave up */
#define QIS_ERR_CAPACITY (-5)     /* a per-search survivor buffer overflowed (raise survivor_cap) */
#define QIS_ERR_STATE (-6)        /* call out of order (e.g. iterate before init_states) */

/* Arithmetic of the local fields and candidate energies (precision modes). The names of the two
 * exact modes are historical (a BF16 hi/lo split and an FP8 digit were planned); what they do on
 * this GPU is stated beside each. */
#define QIS_FP64 0        /* plain form: FP64 fields, energies and comparisons, in one fixed
                             evaluation order (f_i summed with j ascending, E' = E_p + dE) */
#define QIS_SPLIT_BF16 1  /* exact fixed point: J and h on the grid 2^-q (Jq = J 2^q, int64);
                             Jq written in balanced base-4096 digits (12-bit, |d| <= 2048; 11-bit
                             digits, base 2048, above a padded n of 8192), each an exact FP16
                             integer; fields from one FP16 tensor-core GEMM per digit with FP32
                             accumulation, exact for any summation order, combined in int64;
                             FP32 candidate filter with a rigorous error band; exact int64 keys */
#define QIS_PM1_FP8 2     /* integer couplings |J_ij| <= 15 (e.g. +-J) and integer h: q = 0 and one
                             FP16 digit, the same exact integer fields and energies */

typedef struct qis_ctx qis_ctx; /* opaque, library-owned */

typedef struct {
  int K;             /* each search keeps K+1 states (Alg. 2 requires 1 <= K < 2^n) */
  int R;             /* searches (initial states) per instance: L of Alg. 4 */
  int precision;     /* QIS_FP64 | QIS_SPLIT_BF16 | QIS_PM1_FP8 */
  int max_n;         /* largest n of any instance added to this context (2 <= n <= 16384) */
  int max_instances; /* capacity of the instance table */
  int survivor_cap;  /* per-search candidate buffer (0 = default 2048) */
  int device;        /* CUDA device ordinal */
  uint64_t seed;     /* key of the library's SplitMix64 stream for random initial states */
  int flips;         /* flip set of every search: QIS_FLIPS_SINGLE_PAIR (0, default), QIS_FLIPS_SINGLE
                        or QIS_FLIPS_EXCHANGE */
} qis_config;

/* Flip sets (the candidates generated from a parent):
 *   QIS_FLIPS_SINGLE_PAIR  single flips X_i and pair flips X_i X_j (Eq. (H1), the paper's study);
 *   QIS_FLIPS_SINGLE       single flips only (J = 1: the uniform transverse field of the
 *                          Sec. V outlook);
 *   QIS_FLIPS_EXCHANGE     spin exchanges only (the XX + YY interaction of the Sec. V outlook):
 *                          pairs (i, j) with s_i != s_j, so every kept state has the initial
 *                          state's magnetisation; a search whose sector holds fewer than K+1
 *                          states stops once all of them are used.
 * Candidate indices keep the default numbering (c = i, c = n + rank(i, j)); excluded candidates
 * are skipped. */
#define QIS_FLIPS_SINGLE_PAIR 0
#define QIS_FLIPS_SINGLE 1
#define QIS_FLIPS_EXCHANGE 2

/* Create a context and allocate every device buffer it will use (sized by max_n,
 * max_instances, K, R). Nothing else allocates device memory afterwards. */
int qis_create(const qis_config* cfg, qis_ctx** out);

/* Free the context and all its device memory. NULL is ignored. */
void qis_destroy(qis_ctx* ctx);

/* Message of the last failing call on this context (or of the last failed qis_create
 * when ctx is NULL). Never NULL; valid until the next call on the context. */
const char* qis_last_error(const qis_ctx* ctx);

/* Add one Ising instance H0 (Eq. (1)).
 *   n: number of spins, 2 <= n <= cfg.max_n.
 *   J: n*n FP64 row-major, symmetric (bitwise J_ij == J_ji), zero diagonal, finite; host
 *      memory (not retained). In the split modes a page-locked J (cudaHostAlloc /
 *      cudaHostRegister) is read by the device directly, without a staging copy.
 *   h: n FP64 finite, host memory.
 * Instances get consecutive ids from 0. In QIS_SPLIT_BF16 the values are represented on
 * the grid 2^-q with the smallest q that holds them exactly, capped so that every energy
 * sum stays below 2^52 * 2^-q; if the cap binds, J and h are rounded to that grid and
 * qis_instance_info reports it. QIS_PM1_FP8 requires integer J (|J_ij| <= 15) and h.
 * Synchronises the library stream (validation result). */
int qis_create_instance(qis_ctx* ctx, int n, const double* J, const double* h, int* instance_id);

/* Add `count` instances at once (Eq. (1)), as `count` calls of qis_create_instance would, but
 * with one validation read-back for the whole batch: n[k], J[k], h[k] as there; ids
 * (may be NULL) receive the new ids. If any instance is invalid, none of the batch is added
 * and the error names the first. Synchronises the library stream once. */
int qis_create_instances(qis_ctx* ctx, int count, const int* n, const double* const* J, const double* const* h,
                         int* instance_ids);

/* Remove every instance (ids restart at 0); device buffers stay allocated. */
int qis_clear_instances(qis_ctx* ctx);

/* Grid exponent q and number of FP16 digits (12-bit balanced digits, 11-bit above a padded n of
 * 8192) of an instance's fixed-point couplings, and whether its input had to be rounded onto the
 * grid (QIS_SPLIT_BF16 / QIS_PM1_FP8; q = -1 and 0 digits in QIS_FP64). */
int qis_instance_info(qis_ctx* ctx, int instance_id, int* q, int* digits, int* rounded);

/* Number of spins n of an instance (e.g. after qis_load); QIS_ERR_INVALID_ARG for an id
 * that does not exist. */
int qis_instance_n(qis_ctx* ctx, int instance_id, int* n);

/* Set the R initial states of an instance and reset its R searches to the start of
 * Alg. 3: list = [initial state] followed by K empty slots, nothing used.
 *   bits: R*W words (search r's state at bits + r*W), or NULL to draw every bit from the
 *         library's SplitMix64 stream: bit i of search r of instance id is the top bit of
 *         value (r*n + i) of the stream keyed by key(seed, id), i.e. rand_between(0, 2^n-1)
 *         of Alg. 4.
 * The searches start (initial energies, lists) with one launch for every instance set since,
 * at the next call that reads or advances them; the caller's buffer is free on return. When
 * that call is qis_iterate with at least one iteration of the fused search kernel (the exact
 * modes with a padded n up to 1024), the initial energies are formed in the first iteration
 * from the initial states' exact local fields, E = (sum_i s_i f_i + sum_i s_i h_i) / 2 (Eq. 1
 * with f = J s + h), which that iteration computes anyway; every other call forms them by a
 * separate rescoring launch. Both give the same exact value. */
int qis_init_states(qis_ctx* ctx, int instance_id, const uint64_t* bits);

/* Reset every search of every instance to its stored initial state (device-side, no host
 * copy): the searches restart, as after qis_init_states, at the next call that reads or
 * advances them. Also clears the device error flags (timeout, survivor overflow) of earlier
 * iterations. */
int qis_reset(qis_ctx* ctx);

/* Run n_iters iterations of Alg. 3 on every search of every instance (lockstep).
 * A search whose kept states are all used does nothing in an iteration.
 *   n_active: if not NULL, receives the number of searches that still have an unused
 *             state after the last iteration (this synchronises the stream).
 * Device-side failures (survivor overflow, bounded-wait timeouts) are reported by this
 * or the next synchronising call. */
int qis_iterate(qis_ctx* ctx, int n_iters, int* n_active);

/* Kept list of one search r (0 <= r < R) of an instance, in key order (diagnostics,
 * parity tests, checkpoints). Outputs hold K+1 entries; entries past *count are
 * undefined. Any output pointer may be NULL. */
int qis_search_list(qis_ctx* ctx, int instance_id, int r, uint64_t* bits, double* E,
                    uint8_t* used, uint64_t* stamp, int* count);

/* Replace the kept list of search r of an instance (the inverse of qis_search_list): used
 * to merge lists computed elsewhere (another process or GPU running other searches of the
 * same instance) with the device's Alg. 4 merge, and by qis_load.
 *   count: entries, 1 <= count <= K+1; bits: count*W words (bit i = sigma_i, bits above n
 *   zero), states distinct; E: count finite energies, nondecreasing (the list order of
 *   Alg. 2); used: count flags (l of Alg. 3) or NULL for all false; stamp: count arrival
 *   keys (t << 32 | candidate index) or NULL for 0..count-1; t: iterations already done.
 * The search becomes active when some entry is unused. The energies are taken as given.
 * Synchronises; QIS_ERR_INVALID_ARG on any violated condition, the list then unchanged. */
int qis_set_search_list(qis_ctx* ctx, int instance_id, int r, int count, const uint64_t* bits,
                        const double* E, const uint8_t* used, const uint64_t* stamp, int t);

/* Checkpoint of the whole search state: every instance (J, h), its R initial states and
 * every search's kept list with its used flags, stamps, iteration counter and active flag,
 * followed by a 64-bit FNV-1a checksum. Synchronises. A failed write removes the file. */
int qis_save(qis_ctx* ctx, const char* path);

/* Resume from a qis_save file into a context that has no instances yet and was created
 * with the same K, R and precision (max_n and max_instances large enough). Iterating the
 * loaded context continues the saved searches exactly as the saved context would have.
 * QIS_ERR_INVALID_ARG for a missing, truncated or corrupted file (checksum) or a config
 * mismatch; QIS_ERR_STATE if the context already holds instances. */
int qis_load(qis_ctx* ctx, const char* path);

/* Alg. 4 merge of the R lists of an instance followed by rescoring: the first
 * min(k, count) states of the union of the R lists (each state at its first occurrence
 * in search order), ordered by (E, search index, position in that search's list).
 *   bits_out: k*W words; E_out: k energies recomputed from scratch from J, h (Eq. (1)): in
 *             exact integer arithmetic for an instance on its grid 2^-q in the split modes
 *             (the value of any FP64 summation of those grid numbers), else in FP64;
 *   src_out (may be NULL): (r << 32) | position of each state's first occurrence;
 *   n_out: number of states written. */
int qis_topk_states(qis_ctx* ctx, int instance_id, int k, uint64_t* bits_out, double* E_out,
                    uint64_t* src_out, int* n_out);

/* qis_topk_states for every instance at once (one merge, one rescoring launch, one copy):
 *   bits_out: n_inst*k*Wmax words, state r of instance i at (i*k + r)*Wmax (Wmax = words of
 *             max_n; words past the instance's own W are zero);
 *   E_out, src_out (each may be NULL): n_inst*k values, entry i*k + r;
 *   n_out (may be NULL): n_inst counts, min(k, merged count of instance i).
 * 0 <= k <= K+1. Synchronises. */
int qis_topk_states_all(qis_ctx* ctx, int k, uint64_t* bits_out, double* E_out, uint64_t* src_out, int* n_out);

/* Alg. 4 merge of every instance on the device, asynchronously, into a library buffer
 * that the next qis_topk_states reads without merging again. */
int qis_merge(qis_ctx* ctx);

/* FP64 energies (Eq. (1)) of `count` caller states of an instance, computed on the GPU. */
int qis_energies(qis_ctx* ctx, int instance_id, int count, const uint64_t* bits, double* E_out);

/* Block until all device work of the context is done; reports deferred device errors. */
int qis_synchronize(qis_ctx* ctx);

/* Bound of every device-side wait of the context's kernels (the mbarrier waits of the tensor-core
 * field GEMM and of the dense pair scan's staging ring), in ns of %globaltimer (2 s by default;
 * 1e3 <= limit_ns <= 6e10). A wait that runs out sets the context's timeout flag, reported as
 * QIS_ERR_DEVICE_TIMEOUT by the next synchronising call; the kernel then waits (at most 2 s) for
 * the copies and tensor-core operations it already issued, frees its tensor memory and returns,
 * so the context stays usable: qis_reset clears the flag and restarts the searches.
 * probe = 1 makes every later field GEMM first wait on a barrier that nothing ever completes, so
 * that path can be exercised without any fault (failure-detection tests); 0 for normal work. */
int qis_set_wait_limit(qis_ctx* ctx, uint64_t limit_ns, int probe);

/* Launch statistics: number of kernels this context has launched so far. */
int qis_kernel_launches(qis_ctx* ctx, uint64_t* count);

/* Candidates decided since the context was created, per expanded parent: pairs n(n-1)/2 and
 * singles n (QIS_FLIPS_SINGLE_PAIR, the Sec. III flip sets), singles n only (QIS_FLIPS_SINGLE),
 * pairs n_up n_down only (QIS_FLIPS_EXCHANGE). Synchronises the stream. */
int qis_candidate_count(qis_ctx* ctx, uint64_t* pairs, uint64_t* singles);

/* Launch shapes of the iteration. None of them changes any result (the candidate sets, the
 * survivor decisions and the exact keys are the same for every setting); they only trade
 * parallelism against reuse.
 *   scan_chunk_nc: the pair scan covers each 32-row block with column chunks of 32*NC sites,
 *                  NC <= scan_chunk_nc (1..8; default 8);
 *   scan_search_group: searches of an instance per scan task (0 = all R; smaller groups
 *                  give more, shorter tasks for few instances);
 *   gemm_tile_searches: searches per tensor-core tile of the local-field GEMM (multiple of
 *                  16, at most 256, digits * it <= 512; 0 = automatic);
 *   pair_scan:     which form of the split modes' FP32 pair filter runs: 1 = output-sensitive
 *                  (one block per search: the live rows c_i >= RD(min_j a_j - rm_i), with
 *                  rm_i = max_j |4J~_ij|, and each live row's prefix of the columns sorted by
 *                  a_j; needs a padded size of at most 4096), run inside the fused search
 *                  kernel where it can (one block per search takes it through every iteration of
 *                  a qis_iterate call: padded n <= 1024, K+1 <= 256, fields by update; the
 *                  environment variable QIS_FUSED=0 turns the fused kernel off), else as its own
 *                  kernel in every iteration; 3 = output-sensitive, always as its own kernel in
 *                  every iteration (the per-kernel form); 2 = dense register tiles (shaped by
 *                  scan_chunk_nc and scan_search_group); 0 = automatic (1 where allowed, else 2;
 *                  the environment variable QIS_DENSE_SCAN=1 makes 2 the default).
 *                  Every form gives the same kept lists. QIS_FP64 scans every pair in its plain
 *                  FP64 form whatever this says; qis_get_tuning reports 2 there. */
typedef struct {
  int scan_chunk_nc;
  int scan_search_group;
  int gemm_tile_searches;
  int pair_scan;
} qis_tuning;

/* Current launch shapes (automatic values resolved). */
int qis_get_tuning(qis_ctx* ctx, qis_tuning* out);

/* Set the launch shapes for the current and later instances. QIS_ERR_INVALID_ARG for values
 * out of range, pair_scan 1 or 3 where the output-sensitive scan cannot run (QIS_FP64, padded size
 * above 4096) or a scan task list larger than the context holds (the setting is unchanged). */
int qis_set_tuning(qis_ctx* ctx, const qis_tuning* t);

/* Autotuner: times `iters` iterations from the initial states for candidate launch shapes
 * (coordinate search over chunk width, search group and GEMM tile, each timed after one
 * untimed run) and keeps the fastest. Every search is reset to its initial state afterwards
 * (as qis_reset). best / best_ms (may be NULL) receive the choice and its time. */
int qis_autotune(qis_ctx* ctx, int iters, qis_tuning* best, double* best_ms);

/* Local fields by update (Sec. III energy algebra; the incremental form of the fields): a kept
 * state is a one- or two-site flip of the parent it was generated from, so its exact integer
 * fields are that parent's minus the flipped sites' coupling columns, O(n) instead of the
 * O(n^2) field GEMM. The context keeps the fields of the last ring_n parents of every search
 * (as many iterations as fit in 4 GiB, 2 to 128); a parent whose generator is older, the
 * initial state and the entries of an imported list get full fields from the tensor-core GEMM
 * (its tiles holding no such parent are skipped). Results are bit-identical either way.
 * on = 1 (the default in the split modes) or 0; QIS_ERR_INVALID_ARG for on = 1 in the FP64
 * mode (its fields follow the defining FP64 summation order) or with the SIMT field kernel. */
int qis_set_incremental_fields(qis_ctx* ctx, int on);

/* Pair terms the candidate scan evaluated one by one since the context was created: in the
 * split modes the scan skips every row whose bound c_i = thr - a_i lies below a lower bound
 * of all its pair terms, and counts (rows evaluated) x (chunk width, masked entries
 * included); in QIS_FP64 every pair is evaluated (the qis_candidate_count pairs). The pairs
 * of qis_candidate_count are all decided exactly either way. The output-sensitive scan
 * (pair_scan 1) counts the pairs it tests one by one (those in the live rows' prefixes, each
 * once). Synchronises the stream. */
int qis_evaluated_pairs(qis_ctx* ctx, uint64_t* pairs);

/* Survivors of the candidate filters (singles and pairs passing the FP32 test with its band)
 * that the merge read, summed over every search and iteration since the context was created:
 * the candidates whose energies the merge computed exactly (Alg. 2's evaluation of the kept
 * candidates). Synchronises the stream. */
int qis_survivor_count(qis_ctx* ctx, uint64_t* count);

/* The library's CUDA stream (a cudaStream_t), so callers can order their own work and
 * CUDA events with respect to the library's kernels. */
int qis_get_stream(qis_ctx* ctx, void** stream);

/* Kernel timing with CUDA events. While enabled, each kernel launched by qis_iterate is
 * bracketed by two events on the library stream. qis_profile_query synchronises, returns the
 * summed device time (ms) and launch count of one kernel class since the last query, and
 * resets that class. Classes: 0 parent pick, 1 local fields, 2 per-search bound,
 * 3 candidate scan, 4 exact merge, 5 fused search kernel (bound, scan and merge of every
 * iteration of a qis_iterate call, and the pick and fields of all but its first). */
int qis_profile_enable(qis_ctx* ctx, int on);
int qis_profile_query(qis_ctx* ctx, int kernel_class, double* total_ms, uint64_t* launches);

/* ------------------------------------------------------------------------------------------
 * Learned warm start. Alg. 4 starts every search from rand_between(0, 2^N - 1); a per-site
 * network can propose the initial states instead. Features of site i (FP64, then FP32):
 * h_i, sum_j J_ij / sqrt(n), sum_j |J_ij| / n, sqrt(sum_j J_ij^2 / n), max_{j!=i} J_ij,
 * min_{j!=i} J_ij, sum_j J_ij h_j / sqrt(n), sum_j J_ij sign(h_j) / sqrt(n). Network:
 * 8 -> hidden -> hidden -> hidden -> 1 with ReLU, BF16 weights (rounded from an FP32 master
 * copy), FP32 accumulation; output z_i = logit of P(s_i = +1); loss: mean binary
 * cross-entropy; training: Adam (beta 0.9 / 0.999, eps 1e-8) on the GPU. Parameters are
 * flattened as W1 (8 x H, row-major), b1 (H), W2 (H x H), b2, W3 (H x H), b3, w4 (H), b4 (1).
 * Pointers are host pointers. */
typedef struct qis_mlp qis_mlp;
typedef struct {
  int hidden;     /* H, multiple of 16 in [16, 1024] */
  int max_sites;  /* capacity of the training set (sites, summed over examples) */
  int batch;      /* training batch (sites) */
  int max_n;      /* largest instance */
  int device;
  uint64_t seed;  /* SplitMix64 key of the He initialisation */
} qis_mlp_config;
int qis_mlp_create(const qis_mlp_config* cfg, qis_mlp** out);
void qis_mlp_destroy(qis_mlp* m);
const char* qis_mlp_last_error(const qis_mlp* m);
int qis_mlp_num_params(qis_mlp* m, int* count);
int qis_mlp_get_params(qis_mlp* m, float* flat);
int qis_mlp_set_params(qis_mlp* m, const float* flat);           /* also resets Adam state */
/* features of the n sites of (J, h): X_out n x 8 */
int qis_mlp_features(qis_mlp* m, int n, const double* J, const double* h, float* X_out);
/* one training example: the sites of (J, h) labelled by the state `bits` (y_i = 1 <=> s_i = +1) */
int qis_mlp_add_example(qis_mlp* m, int n, const double* J, const double* h, const uint64_t* bits);
int qis_mlp_clear_examples(qis_mlp* m);
/* logits of M feature rows (M <= max(batch, max_n)) */
int qis_mlp_forward(qis_mlp* m, int M, const float* X, float* z_out);
/* mean loss and its gradient (flattened as above) on M labelled rows; no update */
int qis_mlp_loss_grad(qis_mlp* m, int M, const float* X, const float* y, double* loss, float* grad_out);
/* `epochs` passes over the training set in batches; final_loss = mean batch loss of the last */
int qis_mlp_train(qis_mlp* m, int epochs, float lr, double* final_loss);
/* Initial states of the R searches of an instance from the network (replacing Alg. 4's
 * rand_between): search 0 takes s_i = +1 iff z_i >= 0; search r >= 1 sets s_i = +1 with
 * probability sigmoid(z_i), drawing value (r*n + i) of the SplitMix64 stream keyed by
 * splitmix64(key(seed, id) ^ 5, 0) (key of qis_init_states). Then as qis_init_states. */
int qis_init_states_learned(qis_ctx* ctx, int instance_id, qis_mlp* m);

/* ------------------------------------------------------------------------------------------
 * Allocation-free candidate selection (the paper has no counterpart; this is a service for
 * callers that cannot allocate device memory when they need the work done: code running
 * while a stream is being captured into a CUDA graph, real-time loops that must not block in
 * the CUDA allocator, plugins whose process owns device memory through another pool).
 *
 * For one parent state psi of an n-spin instance it evaluates every single flip and every
 * pair flip with the library's FP64 arithmetic (E' = E(psi) + dE, as in QIS_FP64) and writes
 * the k candidates of lowest (E', c), ascending, c the candidate index of the conventions
 * above. Unlike every other entry point, all pointers here are DEVICE pointers owned by the
 * caller:
 *   J      n*n FP64 row-major (symmetric, zero diagonal; not validated here)
 *   h      n FP64
 *   bits   ceil(n/64) words of the parent state
 *   E_out  k FP64 energies, c_out k candidate indices, Ep_out (may be NULL) E(psi)
 *   stream a cudaStream_t (NULL = legacy default stream); the call is asynchronous on it.
 * Limits: 2 <= n <= 512, 1 <= k <= min(128, n(n+1)/2); larger sizes return
 * QIS_ERR_INVALID_ARG (message in qis_last_error(NULL)). No device memory is allocated:
 * the scratch space (about 100 KB) is a static array of the library that every GPU which
 * loads the library holds until the process exits. The first call on a device looks up that
 * array's device address, so make the first call before any stream capture. All calls on a
 * device share the array; calls whose kernels may overlap on the GPU must be ordered by the
 * caller (same stream or events), or they race. */
int qis_select_candidates_noalloc(int n, const double* J, const double* h, const uint64_t* bits, int k,
                                  double* E_out, uint32_t* c_out, double* Ep_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* QIS_H */
