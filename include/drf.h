/*
 * drf.h -- C ABI of the B300 data-race-freedom checker for memory access
 * protocols (MAPs).
 *
 * A memory access protocol (paper: "Provable GPU Data-Races in Static Race
 * Detection", PLACES 2022, Fig. 1 "Syntax of MAPs") abstracts a GPU kernel
 * into the array accesses each thread makes: reads rd A[n] and writes
 * wr A[n] whose indices n are integer expressions of the thread id `tid`,
 * loop variables and parameters, inside conditionals, unsynchronized loops
 * (forU) and synchronized loops (forS) whose bodies may contain the barrier
 * `sync`.  Every thread runs the protocol with its own tid (rule par, Fig. 3);
 * the syncs a thread has executed so far number its current phase.  A
 * protocol is data-race free (Definition 1, Sec. 3) iff no phase has two
 * distinct threads i != j and a cell (array, index) that i writes and j reads
 * or writes.  One behavioural type per array (Sec. 3): accesses to different
 * arrays never conflict.
 *
 * This library decides that predicate exactly and concretely for a given
 * thread count, array sizes and parameter values, on the GPU: every thread
 * and every loop iteration is enumerated.  It returns the verdict and, for a
 * racy protocol, the lexicographically smallest witness
 * (phase, array, index, i, j) with i < j.
 *
 * Conventions for every function below:
 *   - The return value is a status: DRF_OK (0) or a negative DRF_E_* code.
 *     A result struct is meaningful only when its own `status` is DRF_OK.
 *   - Pointers are host pointers unless a comment says "device".
 *   - The caller owns every buffer it passes in; the library copies what it
 *     needs before returning and never keeps a caller pointer.
 *   - Streams are passed as `void*` holding a cudaStream_t; NULL means the
 *     context's own stream.
 *   - A context is not thread-safe: use one per host thread, or the server
 *     functions (which are).
 *
 * Protocol text syntax (compiled by drf_protocol_compile):
 *   program := decl* stmt*
 *   decl    := "array" NAME ("," NAME)* ";"  |  "param" NAME ("," NAME)* ";"
 *   stmt    := "skip" ";" | "sync" ";" | ("rd" | "wr") NAME "[" expr "]" ";"
 *            | "if" "(" cond ")" "{" stmt* "}" ["else" "{" stmt* "}"]
 *            | ("forU" | "forS") NAME "in" expr ".." expr "{" stmt* "}"
 *   expr    := integer | "tid" | NAME | expr (+ - * / %) expr | "-" expr
 *            | "min(" expr "," expr ")" | "max(" expr "," expr ")" | "(" expr ")"
 *   cond    := "true" | "false" | expr (== = != < <= > >=) expr
 *            | cond "&&" cond | cond "||" cond | "!" cond | "(" cond ")"
 * Arrays and parameters are numbered in declaration order; their sizes and
 * values come from drf_bounds at check time.  `forU x in lo .. hi` runs
 * x = lo, ..., hi-1 (rules for-1 / for-2, Fig. 3).  `sync` and `forS` may only
 * appear in the synchronized fragment: at top level or inside forS bodies,
 * never inside forU or if bodies (Fig. 1).  A loop variable may not rebind a
 * name in scope (rule t-for, Fig. 4).  `/` is floor division and `%` the
 * Euclidean remainder (always in [0, |divisor|)).
 */
#ifndef DRF_H
#define DRF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status -- */
#define DRF_OK                   0
#define DRF_E_INVALID_ARG       -1   /* null pointer, count mismatch, bad option */
#define DRF_E_PARSE             -2   /* protocol text does not parse */
#define DRF_E_INVALID_BYTECODE  -3   /* malformed or truncated bytecode */
#define DRF_E_UNBOUND_VAR       -4   /* a name that is not tid, a parameter or an enclosing loop variable (rule t-n) */
#define DRF_E_UNKNOWN_ARRAY     -5   /* access to an undeclared array */
#define DRF_E_REBIND            -6   /* loop variable rebinds a name in scope, or a duplicate declaration */
#define DRF_E_SYNC_IN_UNSYNC    -7   /* sync or forS inside forU / if (Fig. 1) */
#define DRF_E_OVERFLOW_RISK     -8   /* some intermediate value may leave int64 (interval analysis) */
#define DRF_E_INDEX_OOB         -9   /* an evaluated index is outside [0, cells) */
#define DRF_E_DIV_ZERO         -10   /* division or remainder by zero */
#define DRF_E_KEY_TOO_WIDE     -11   /* phase+array+index+tid bits exceed the 64-bit access key */
#define DRF_E_NOMEM            -12   /* device or host allocation failed */
#define DRF_E_CUDA             -13   /* a CUDA runtime call failed */
#define DRF_E_TIMEOUT          -14   /* a bounded device-side wait gave up, or a poll timed out */
#define DRF_E_BUSY             -15   /* server queue full / server not running */
#define DRF_E_LIMIT            -16   /* a size limit of this implementation (nesting, items, threads) */
#define DRF_E_NOT_FOUND        -17   /* unknown server ticket */
#define DRF_E_INTERNAL         -18   /* an internal consistency check failed */

/* verdicts (drf_result.verdict) */
#define DRF_VERDICT_DRF                 0
#define DRF_VERDICT_RACY                1
#define DRF_VERDICT_BARRIER_DIVERGENCE  2

/* ------------------------------------------------------------------ types -- */
typedef struct drf_ctx drf_ctx;      /* device buffers, streams, tuning state */
typedef struct drf_plan drf_plan;    /* a fixed batch prepared for repeated launches */

/* Bounds a protocol is checked under.  loc_cells[l] is the size of array l
 * (declaration order, nlocs entries); params[k] the value of parameter k. */
typedef struct {
    uint32_t nthreads;           /* thread ids 0 .. nthreads-1 */
    uint32_t nlocs;              /* must equal the protocol's array count */
    const uint64_t *loc_cells;   /* host, nlocs entries */
    uint32_t nparams;            /* must equal the protocol's parameter count */
    const int64_t *params;       /* host, nparams entries */
} drf_bounds;

/* Result of one check.
 *   status != DRF_OK: an evaluation error (DRF_E_INDEX_OOB, DRF_E_DIV_ZERO)
 *     or a rejection; for evaluation errors err_tid is the smallest failing
 *     thread and err_ordinal the number of accesses it completed first.
 *   verdict RACY: the lexicographically smallest (phase, loc, index, tid_i,
 *     tid_j) with tid_i < tid_j both accessing cell (loc, index) in `phase`
 *     and at least one writing; i_writes / j_writes say which do.
 *   verdict BARRIER_DIVERGENCE: threads ran different numbers of syncs;
 *     div_tid is the smallest thread whose count differs from thread 0's.
 *   tuples: dynamic accesses of all threads; phases: 1 + syncs of thread 0
 *   (0 when nthreads is 0). */
typedef struct {
    int32_t status;
    int32_t verdict;
    uint32_t phase, loc;
    uint64_t index;
    uint32_t tid_i, tid_j;
    uint32_t i_writes, j_writes;
    uint32_t div_tid, sync_count_0, sync_count_div;
    uint32_t phases;
    uint64_t tuples;
    uint32_t err_tid, reserved0;
    uint64_t err_ordinal;
} drf_result;

/* Context options (all zero = defaults). */
typedef struct {
    uint32_t radix_bits;         /* sort path's radix digit width 4..8; 0 = 8, or tuned by plans
                                    with DRF_OPT_AUTOTUNE (drf_plan_config) */
    uint32_t flags;              /* DRF_OPT_* */
    uint64_t max_device_bytes;   /* cap on the context's device workspace; 0 = none */
} drf_opts;

#define DRF_OPT_PROFILE_STAGES 0x1u   /* record per-kernel CUDA events in plans */
#define DRF_OPT_AUTOTUNE       0x2u   /* plans: time candidate launch configurations, keep the fastest */
/* Back end (at most one; neither = chosen per batch).  Both decide
 * Definition 1 exactly and return identical results:
 *   sort path   -- one 64-bit key per access (phase, array, index, tid, mode),
 *                  radix-sorted on the cell fields, racy segments detected;
 *                  with the range pieces planned (see DRF_OPT_RANGE_ANY) the
 *                  range accesses' keys are written from the pieces, one per
 *                  distinct (thread, offset) (drf_plan_keys);
 *   owner table -- one 32-bit record per (phase, array, index) cell, rows
 *                  up to the static bound on syncs: the first accessor, "a
 *                  second thread accessed it", "it was written"; a cell is
 *                  racy iff written with a second thread, and a further pass
 *                  restricted to the first racy cell finds the witness
 *                  threads.  It needs (sync bound + 1) x (sum of array
 *                  sizes) x 4 bytes, at most 64 GiB.
 * The automatic choice takes the owner table when it fits and is at most
 * max(256 MiB, 256 bytes per access tuple); otherwise, or when the table
 * cannot be allocated, the sort path.  Forcing the owner table on a batch
 * it cannot hold returns DRF_E_LIMIT (or DRF_E_NOMEM). */
#define DRF_OPT_PATH_SORT      0x4u
#define DRF_OPT_PATH_TABLE     0x8u
/* Plans over a single protocol may run kernels specialized to it: its
 * count, owner-table and witness passes translated to CUDA C (loops as
 * loops, every coefficient, array size and table stride a constant) and
 * compiled for sm_103a with NVRTC at plan creation (about 0.1 - 1 s); the
 * results are those of the interpreter.  Without DRF_OPT_AUTOTUNE such a
 * plan uses them whenever they compile; with it the tuner times them
 * against the interpreted configurations.  Plans keep the interpreter when
 * NVRTC is unavailable or the protocol has no owner table.
 * drf_check / drf_check_batch of a single protocol on such a context use
 * kernels specialized to it too when the protocol may make 2^21 accesses or
 * more (smaller checks run faster interpreted than the compile would take),
 * kept per context and keyed by the bytecode and bounds (at most 32
 * protocols, then the cache starts over): the first check of a protocol
 * under given bounds compiles them (that call takes the compile time), later
 * ones reuse them; every check still validates, lowers and uploads the
 * protocol and runs every pass.  Protocols the automatic choice would not
 * give the owner table, and forced sort-path contexts, keep the
 * interpreter. */
#define DRF_OPT_SPECIALIZE     0x10u
/* The range pieces for batches of any size, checked by any entry point:
 * the owner table's range pass (drf_plan_specialized), or on a forced sort
 * path the range accesses' keys written from the pieces.  By default plans and single-protocol
 * checks take it when its range accesses make 2^22 access tuples or more
 * (below that, planning its work lists, uploading them and the extra kernel
 * cost more than the table pass they relieve; a repeated drf_check of one
 * protocol plans it once), and checks of several protocols at once and the
 * server's rounds do not (the host planning of a batch checked once, about
 * 0.1 ms per protocol, costs more than the device time it saves).  Results
 * are the same either way. */
#define DRF_OPT_RANGE_ANY      0x20u

#define DRF_PATH_SORT  1
#define DRF_PATH_TABLE 2

/* ------------------------------------------------------- library / errors -- */

/* Library ABI version (this header: 1). */
int drf_version(void);

/* Static name of a status code ("DRF_E_INDEX_OOB", ...). */
const char *drf_status_string(int status);

/* --------------------------------------------------------------- contexts -- */

/* Creates a context on CUDA device `device` (the library calls
 * cudaSetDevice(device) on every entry that touches the GPU).  opts may be
 * NULL.  *out receives the context; release it with drf_ctx_destroy. */
int drf_ctx_create(int device, const drf_opts *opts, drf_ctx **out);

/* Waits for the context's work, frees its device memory and streams. */
void drf_ctx_destroy(drf_ctx *ctx);

/* Message for the context's last failed call ("" if none).  Valid until the
 * next call on the same context. */
const char *drf_last_error(const drf_ctx *ctx);

/* ------------------------------------------------------- protocol front-end */

/* Compiles protocol text (syntax above; Fig. 1 with the synchronized fragment
 * admitting accesses) into the library's portable bytecode.  On success
 * *bytecode is a malloc'd buffer of *len bytes (free with drf_free).  On
 * failure returns DRF_E_PARSE / _UNBOUND_VAR / _UNKNOWN_ARRAY / _REBIND /
 * _SYNC_IN_UNSYNC and writes a message into err (errlen bytes, may be 0).
 * Host only; no GPU needed. */
int drf_protocol_compile(const char *text, uint8_t **bytecode, size_t *len,
                         char *err, size_t errlen);

/* BabyCUDA front-end (Sec. 3, Fig. 3 syntax; typing rules of Fig. 4).
 * Reads a BabyCUDA program --
 *   stmt := "let" NAME "=" ARRAY "[" expr "]" ";"     (read; NAME holds the value)
 *         | ARRAY "[" expr "]" ":=" expr ";"          (write of a payload)
 *         | "if" "(" cond ")" "{" stmt* "}" ["else" "{" stmt* "}"]
 *         | ("for" | "forS") NAME "in" expr ".." expr "{" stmt* "}"
 *         | "sync" ";" | "skip" ";"
 * with the same declarations and expressions as protocol text -- and infers
 * its memory access protocol: a write A[n] := m types as wr A[n] (the payload
 * is dropped, rule t-write), "let x = A[n]; b" as rd A[n]; b where x may
 * appear in payloads only (rule t-read keeps x out of the typing
 * environment, so an index, condition or loop bound that depends on data
 * read from an array is rejected with DRF_E_UNBOUND_VAR -- the paper's
 * eqn. illtyped).  "for" is the unsynchronized loop.  Output and errors as
 * drf_protocol_compile.  Host only. */
int drf_babycuda_infer(const char *text, uint8_t **bytecode, size_t *len, char *err, size_t errlen);

/* MAP text of a bytecode (arrays A0.., parameters P0.., loop variables
 * v<slot>); drf_protocol_compile reads it back to the same bytecode.
 * *text is malloc'd (free with drf_free). */
int drf_protocol_text(const uint8_t *bytecode, size_t len, char **text);

/* Array and parameter counts a bytecode declares (validates it fully). */
int drf_protocol_info(const uint8_t *bytecode, size_t len, uint32_t *nlocs, uint32_t *nparams);

/* Static facts about a protocol under given bounds, from the host-side
 * validation and interval analysis that every check runs first (no GPU):
 * upper bounds on access tuples (all threads) and syncs (one thread), the
 * number of work items each thread is cut into, whether 64-bit arithmetic is
 * needed, and the sorted key bits.  Returns the status a check would return
 * before touching the GPU (DRF_E_OVERFLOW_RISK, DRF_E_LIMIT, ...). */
typedef struct {
    uint64_t tuple_bound;
    uint64_t sync_bound;
    uint32_t items;
    uint32_t wide_arithmetic;
    uint32_t sort_bits;
    uint32_t key_bits;
    /* access tuples the owner table's range pass takes when the protocol is
     * checked alone on the owner-table path: its accesses at a * tid plus a
     * function of the loop variables (|a| <= 64, under a remainder that wraps
     * at most 64 times over the threads), in loops and conditions that do
     * not read tid and hold no sync, applied cell range by cell range in
     * shared memory (0 when it has none or they make under a quarter of its
     * tuples); counted at any size (see DRF_OPT_RANGE_ANY for when checks
     * take the pass) */
    uint64_t range_tuples;
} drf_analysis;

int drf_protocol_analyze(const uint8_t *bytecode, size_t len, const drf_bounds *bounds, drf_analysis *out);

/* Frees memory returned by this library. */
void drf_free(void *p);

/* ------------------------------------------------------------------ checks -- */

/* Checks one protocol (bytecode of `len` bytes) under `bounds` and writes
 * the result to *out.  Runs the whole device pipeline on `stream` and blocks
 * until the result is on the host: the front (count the accesses per thread
 * and work item, scan them into phases and offsets), then the back end the
 * context's options select (DRF_OPT_PATH_*; by default the owner table when
 * it fits, see below): either key emission, radix sort and segmented
 * detection, or the owner-table pass, its scan and the witness pass; then
 * the result.  Returns out->status. */
int drf_check(drf_ctx *ctx, const uint8_t *bytecode, size_t len,
              const drf_bounds *bounds, drf_result *out, void *stream);

/* Checks n protocols in one pass of the device pipeline (the protocol id
 * rides in the top bits of every access key).  out has n entries; each
 * protocol gets its own status, identical to what drf_check returns for it
 * alone.  The call's return value is DRF_OK unless the batch as a whole
 * failed (then no out entry is meaningful). */
int drf_check_batch(drf_ctx *ctx, uint32_t n, const uint8_t *const *bytecodes,
                    const size_t *lens, const drf_bounds *bounds, drf_result *out,
                    void *stream);

/* Bytes the context's last drf_check / drf_check_batch copied host->device
 * (bytecode-derived device programs, items, schedules) and device->host
 * (tuple count, control block, results). */
int drf_ctx_transfer_bytes(const drf_ctx *ctx, uint64_t *h2d, uint64_t *d2h);

/* ---------------------------------------------------- allocation-free check */

/* Size of the fixed device array that drf_check_noalloc works in. */
#define DRF_NOALLOC_SCRATCH_BYTES (64ull << 20)

/* drf_check without any device allocation, for callers that cannot call
 * cudaMalloc when they need a check: a process whose device memory is
 * already reserved by another component's allocator, code that may not
 * allocate after start-up, or a path where an allocation's implicit
 * synchronisation is not acceptable.  (The paper has no counterpart; this
 * is a deployment variant of drf_check.)
 *
 * Every buffer of the pipeline is carved from one file-scope device array
 * of DRF_NOALLOC_SCRATCH_BYTES, reserved when the library's device code is
 * loaded on a GPU and held there until the process exits.  The call works
 * on the current device and `stream` (NULL: the legacy default stream),
 * needs no context, and never calls cudaMalloc, cudaFree or any allocating
 * library routine.  Its result equals drf_check's.
 *   - Every call looks up the array's device address in the current context
 *     (a lookup, no allocation); the first call on a device also loads the
 *     library's device code there, so make that first call before any
 *     stream capture.
 *   - Protocols whose buffers do not fit the array (roughly 3.5 million
 *     access tuples or fewer fit; the exact need depends on the thread
 *     count and work items) are rejected with DRF_E_LIMIT in the return
 *     value and in out->status.
 *   - All calls on a device share the one array and leave their data in it;
 *     each call clears what it needs cleared.  Calls that overlapped on the
 *     GPU would race on the array; the library rules that out within a
 *     process: a per-device lock is held for the whole call, and a call
 *     waits for its own GPU work before it returns, so calls from several
 *     host threads (on any streams) run one after another.  Calls on
 *     different devices use different arrays and run in parallel.
 * Blocks until the result is on the host; returns out->status. */
int drf_check_noalloc(const uint8_t *bytecode, size_t len, const drf_bounds *bounds, drf_result *out,
                      void *stream);

/* ------------------------------------------------------ one protocol, sharded */

/* A protocol's cells split over several checkers (several GPUs, or several
 * calls).  Definition 1 (Sec. 3) decides each (phase, array, index) cell on
 * its own -- a race needs two threads on the same cell in the same phase --
 * so the cells can be partitioned and checked independently; only the
 * results are combined.  Cells are numbered in the witness's lexicographic
 * order, position = phase * (sum of the array sizes) + (the array's offset
 * among them, declaration order) + index, over the phases 0 .. S where S is
 * the static bound on syncs per thread (drf_analysis.sync_bound).  Shard k
 * of n takes positions [k * total / n, (k + 1) * total / n).
 *
 * drf_shard_range: the window [*lo, *hi) of shard `shard` of `nshards` and,
 * when `positions` is not NULL, the total.  Host only (no GPU needed). */
int drf_shard_range(const uint8_t *bytecode, size_t len, const drf_bounds *bounds, uint32_t shard, uint32_t nshards,
                    uint64_t *lo, uint64_t *hi, uint64_t *positions);

/* Checks shard `shard` of `nshards` of one protocol on the context's GPU:
 * every thread is evaluated (evaluation errors, sync counts, barrier
 * divergence and the tuple count are facts of the whole protocol, identical
 * in every shard), but only the shard's cells are recorded in the owner
 * table, so *out reports RACY iff the shard holds a racy cell, with the
 * lexicographically smallest one and its witness threads (computed from all
 * threads' accesses to that cell).  Always the owner-table back end
 * (interpreted); DRF_E_LIMIT when the protocol's table does not fit. */
int drf_check_shard(drf_ctx *ctx, const uint8_t *bytecode, size_t len, const drf_bounds *bounds, uint32_t shard,
                    uint32_t nshards, drf_result *out, void *stream);

/* Combines the n shard results of one protocol (any order) into the result
 * drf_check gives for it: the shards must agree on every fact of the whole
 * protocol (status, error thread and ordinal, tuples, phases, sync counts,
 * divergence) -- else DRF_E_INTERNAL; an error or a divergence is then the
 * result; otherwise the racy shard result with the smallest (phase, array,
 * index), or DRF if none is racy.  Host only: a min-reduction over records
 * of a few dozen bytes, the one exchange between the checkers of a
 * protocol's shards. */
int drf_merge_shards(const drf_result *parts, uint32_t n, drf_result *out);

/* Diagnostics: copies the sorted access keys of the context's last
 * drf_check / drf_check_batch into keys (device -> host, at most cap) and
 * sets *n to their number.  layout[0..4] receive the key's field widths:
 * tid, index, array, phase and protocol bits; a key is, from its most
 * significant field down, protocol | phase | array | index | tid | mode
 * (mode 1 = write).  DRF_E_NOT_FOUND when that check ran the owner-table
 * path (which sorts nothing). */
int drf_debug_sorted_keys(drf_ctx *ctx, uint64_t *keys, uint64_t cap, uint64_t *n, uint32_t layout[5]);

/* Test hook for the bounded waits of the radix sort's look-back: the
 * context's next `launches` checks that run the sort path leave tile 0's
 * look-back status unpublished in every radix pass and let each waiting
 * digit give up after 64 waits instead of about a second's worth.  Those
 * checks return DRF_E_TIMEOUT (no verdict) without any GPU fault -- the
 * waits end, every store stays inside the key buffers -- and the context
 * works normally afterwards.  Owner-table launches are not affected. */
int drf_debug_stall_lookback(drf_ctx *ctx, uint32_t launches);

/* A parameter swept over a range in one batched pass: checks the protocol
 * for every value v in [lo, hi) of parameter `param` (the other bounds as
 * given), as a batch of hi - lo protocols -- a bounded stand-in for a
 * symbolic parameter such as M in the paper's Fig. 1.  out has hi - lo
 * entries, out[k] for value lo + k; each equals drf_check at that value. */
int drf_check_param_sweep(drf_ctx *ctx, const uint8_t *bytecode, size_t len, const drf_bounds *bounds,
                          uint32_t param, int64_t lo, int64_t hi, drf_result *out, void *stream);

/* Run-time specialization diagnostics.  Generates the CUDA source of the
 * per-protocol kernels (count, owner-table and witness passes) that a plan
 * over this one protocol compiles with DRF_OPT_SPECIALIZE, and, when
 * `compile` is nonzero, compiles it for sm_103a with NVRTC (no GPU needed).
 * *source receives the text (free with drf_free); log, when not NULL,
 * receives the compiler's log (truncated to loglen).  Returns DRF_E_LIMIT
 * when the protocol cannot be specialized (its owner table does not fit, or
 * more than 64 item shapes), DRF_E_NOT_FOUND when NVRTC cannot be loaded,
 * DRF_E_INTERNAL when NVRTC rejects the source. */
int drf_protocol_specialize(const uint8_t *bytecode, size_t len, const drf_bounds *bounds, int compile,
                            char **source, char *log, size_t loglen);

/* ------------------------------------------------------------------- plans -- */

/* Prepares a fixed batch for repeated checks: validates and lowers every
 * protocol, uploads the device programs, sizes every buffer (one sizing run
 * of the count pass), and records the whole pipeline as a CUDA graph.  A
 * protocol that fails validation or evaluation makes plan creation fail with
 * its status (use drf_check_batch to get per-protocol statuses). */
int drf_plan_create(drf_ctx *ctx, uint32_t n, const uint8_t *const *bytecodes,
                    const size_t *lens, const drf_bounds *bounds, drf_plan **out);

/* Enqueues one complete check of the plan's batch on `stream` (every kernel
 * of the pipeline runs again; nothing is cached between launches) and
 * returns without waiting.  Results stay on the device. */
int drf_plan_launch(drf_plan *plan, void *stream);

/* Waits for the plan's last launch and copies its n results to the host. */
int drf_plan_results(drf_plan *plan, drf_result *out);

/* Statistics of the plan: total access tuples, number of sort passes run,
 * number of kernels one launch runs, sorted key bits. */
int drf_plan_info(const drf_plan *plan, uint64_t *tuples, uint32_t *sort_passes,
                  uint32_t *kernels_per_launch, uint32_t *sort_bits);

/* The keys a sort-path plan sorts per launch (0 on the owner table): the
 * tuples, except that a forced sort path (DRF_OPT_PATH_SORT) emits the
 * range accesses' keys (drf_analysis.range_tuples) once per distinct
 * (thread, offset) -- iterations that repeat an access add no key. */
int drf_plan_keys(const drf_plan *plan, uint64_t *keys);

/* Per-stage device times (milliseconds) of the last launch, when the context
 * was created with DRF_OPT_PROFILE_STAGES: names[i] (static strings) and
 * ms[i] for i < *count (cap entries at most).  Waits for the launch. */
int drf_plan_stage_times(drf_plan *plan, const char **names, float *ms, int cap, int *count);

/* The launch configuration a plan uses: the warp-items per SM its items
 * were cut for (the item-to-warp schedule), the keys per thread of its
 * radix tiles and the radix digit width of its sort (bits per pass; the
 * sort makes ceil(sorted key bits / width) passes).  With DRF_OPT_AUTOTUNE,
 * drf_plan_create times every candidate (granularity 32 / 128 / 512 x tile
 * 12 / 16 / 24 keys per thread, 8-bit digits, on the sort path; granularity
 * x interpreted / specialized on the owner table) on the batch -- each
 * launch after overwriting 256 MiB of scratch, so that it starts with a
 * cold L2 -- then, when a sort-path configuration wins and the context's
 * drf_opts.radix_bits is 0, the same configuration with 6- and 7-bit
 * digits, and keeps the fastest; the choice is cached per workload
 * signature for the process and, when the environment variable
 * DRF_TUNE_CACHE names a file, persisted there.  A nonzero
 * drf_opts.radix_bits fixes the digit width of every sort (it is widened
 * where the key would need more than 8 passes). */
int drf_plan_config(const drf_plan *plan, uint32_t *granularity, uint32_t *radix_items, uint32_t *radix_bits);

/* Whether a plan runs kernels specialized to its protocol
 * (DRF_OPT_SPECIALIZE): *specialized = 0 (no), 1 (yes), 2 (yes, and the
 * protocol's sync structure is the same for every thread and no evaluation
 * can fail, so each item's phase is compiled in and a launch runs neither
 * the count nor the scan pass; the owner-table pass counts the tuples), or
 * 3 (as 2, and the launch runs the range pass: the accesses that
 * drf_analysis.range_tuples counts are applied cell range by cell range in
 * shared memory, the threads reaching a range found as runs of consecutive
 * tids per offset; the owner-table pass applies the other accesses and the
 * range pass merges their records, then finds the first racy cell).
 * Interpreted plans run the range pass too (reported by
 * drf_plan_range_tuples).  When specialization was asked for but not used,
 * log (may be NULL) receives why. */
int drf_plan_specialized(const drf_plan *plan, uint32_t *specialized, char *log, size_t loglen);

/* The back end a plan runs: DRF_PATH_SORT or DRF_PATH_TABLE (see
 * DRF_OPT_PATH_*).  With DRF_OPT_AUTOTUNE the tuner times both back ends
 * (the owner table once per granularity) when the owner table fits. */
int drf_plan_path(const drf_plan *plan, uint32_t *path);

/* The range pass of a plan (zeros when the plan does not run it): *tuples,
 * the access tuples its accesses make in one launch
 * (every thread, every iteration; the owner-table pass applies the other
 * tuples); *updates (may be NULL), the record updates its last launch made
 * -- fewer, since the iterations of an access that share an offset apply
 * the same accesses and are applied once (waits for the launch). */
int drf_plan_range_tuples(const drf_plan *plan, uint64_t *tuples, uint64_t *updates);

/* Releases the plan's device memory and graph. */
void drf_plan_destroy(drf_plan *plan);

/* ----------------------------------------------------------------- server -- */

/* Continuous-batching check server on the context.  Requests submitted from
 * any host thread are admitted into device rounds as device memory (counted
 * from each request's bound on its access tuples) and batch slots allow;
 * up to two rounds overlap on the GPU.  Each result equals drf_check's. */
typedef struct {
    uint64_t max_round_tuples;   /* tuple budget of one round; 0 = default */
    uint32_t max_round_protocols;/* protocols per round; 0 = default */
    uint32_t max_queue;          /* pending requests before submit returns BUSY; 0 = default */
    uint32_t poll_us;            /* an idle worker polls the queue this long (keeping its core
                                    busy) before sleeping: lower latency under moderate load at
                                    the cost of CPU time; at most 10^6; 0 = sleep at once (default) */
    uint32_t reserved;           /* must be 0 */
} drf_server_opts;

int drf_server_start(drf_ctx *ctx, const drf_server_opts *opts);

/* Queues one check (bytecode and bounds are copied).  *ticket identifies it. */
int drf_server_submit(drf_ctx *ctx, const uint8_t *bytecode, size_t len,
                      const drf_bounds *bounds, uint64_t *ticket);

/* Waits up to timeout_us microseconds (negative: forever) for a ticket's
 * result.  DRF_E_TIMEOUT if not done yet; the ticket stays valid.  Once a
 * result has been returned the ticket is released.  latency_ns (may be NULL)
 * receives the time from submit to completion. */
int drf_server_poll(drf_ctx *ctx, uint64_t ticket, drf_result *out, int64_t timeout_us,
                    uint64_t *latency_ns);

/* Counters of the running server: rounds launched, requests completed and
 * the largest number of protocols one round held. */
int drf_server_stats(drf_ctx *ctx, uint64_t *rounds, uint64_t *completed, uint32_t *max_round);

/* Drains in-flight work and stops the server thread. */
int drf_server_stop(drf_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* DRF_H */
