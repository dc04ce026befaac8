/*
 * libvrprpd -- batched candidate evaluation and the searches built on it for
 * the Vehicle Routing Problem with Resource-Constrained Pickup and Delivery
 * (Sodhi, Prasad, Saseendran; arXiv 2602.23685).  One GB300 (sm_103a).
 *
 * Problem (Section 3, "Problem Formulation"): customers C = {1..n}, depot 0,
 * m vehicles of capacity Q (the paper's k), travel times d, processing times
 * p.  Each customer receives one dropoff and one pickup, possibly by
 * different vehicles (Eq. 1); a pickup leaves no earlier than drop + p_c
 * whichever vehicle dropped (Eq. 9); vehicles may not carry fewer than 0 or
 * more than Q resources (Eqs. 13-18); the makespan is the latest return to
 * the depot (Eqs. 21-23).  The library adds a finite depot pool R: the
 * resources all vehicles load at the depot before leaving sum to at most R.
 *
 * Conventions shared by every call
 *  - Op code o = 2c + isPickup for customer c in 1..n (so o in [2, 2n+1]).
 *  - A candidate solution is route-major: ops[off[v] .. off[v+1]) is the
 *    sequence of vehicle v, with off[0] = 0 and off[m] = 2n (Section 4.3,
 *    "tour_v = [(c1,op1),(c2,op2),...]").
 *  - Status bits per candidate (0 = feasible).  A status is not an error.
 *  - Return codes: VRPRPD_OK (0) or a negative error; vrprpd_last_error()
 *    then describes it (per calling thread).
 *  - Pointers are DEVICE pointers unless a parameter says "host".  Calls that
 *    take a stream (a cudaStream_t passed as void*, NULL = legacy default
 *    stream) are asynchronous on that stream; the caller keeps every buffer
 *    alive and unmodified until the stream work completes.  The caller owns
 *    every buffer it passes; the library owns instances and servers until
 *    their *_destroy call.
 */
#ifndef VRPRPD_H
#define VRPRPD_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define VRPRPD_OK 0
#define VRPRPD_EINVAL (-1)   /* bad size, range, alignment or pointer */
#define VRPRPD_ENOMEM (-2)   /* device or host allocation failed */
#define VRPRPD_ECUDA (-3)    /* a CUDA runtime call failed */
#define VRPRPD_ETIMEOUT (-4) /* a bounded device-side wait gave up */
#define VRPRPD_EBUSY (-5)    /* admission refused (server memory budget / slots) */
#define VRPRPD_ENOTREADY (-6)/* request not finished yet */

/* ---- candidate status bits ---- */
#define VRPRPD_CYCLE 1u      /* precedence cycle: some pickup can never follow its drop */
#define VRPRPD_VEH_CAP 2u    /* some vehicle's stock leaves [0, Q] (Eqs. 14, 17, 18) */
#define VRPRPD_POOL 4u       /* start loads exceed the depot pool R */
#define VRPRPD_MALFORMED 8u  /* bad offsets, op codes, or an op missing/duplicated */

/* ---- instance flags ---- */
#define VRPRPD_LOAD_MIN 0u   /* each vehicle loads the least stock its route needs */
#define VRPRPD_LOAD_FULL 1u  /* each vehicle leaves with Q (Eq. 13) */

typedef struct vrprpd_instance vrprpd_instance;

/*
 * Create an instance from integer coordinates (TSPLIB EUC_2D: d(i,j) =
 * nint(sqrt(dx^2 + dy^2)), computed exactly in integers on the device;
 * Section 5.1 uses TSPLIB edge weights as travel times).
 *   coords  host, (n+1) x 2 int32, row 0 is the depot; |coord| <= 2^20.
 *   p       host, n int32 >= 0, p[c-1] is customer c's processing time.
 *   n >= 1, 1 <= m <= 32 for the batched kernels (any m >= 1 for the plain
 *   form), R >= 0, Q >= 1, flags = VRPRPD_LOAD_MIN or VRPRPD_LOAD_FULL.
 * Fails with VRPRPD_EINVAL if (2n+1)*max(d) + n*max(p) exceeds INT32_MAX - 1,
 * the bound under which every schedule time fits int32.  *out receives an
 * instance resident on the current CUDA device.
 */
int vrprpd_instance_create(const int32_t* coords, const int32_t* p, int32_t n, int32_t m,
                           int32_t R, int32_t Q, uint32_t flags, vrprpd_instance** out);

/* Same, from an explicit host (n+1) x (n+1) int32 matrix d >= 0 (row-major,
 * d[i*(n+1)+j] = travel time from i to j; Section 3.1's d_{i,j}). */
int vrprpd_instance_create_dist(const int32_t* d, const int32_t* p, int32_t n, int32_t m,
                                int32_t R, int32_t Q, uint32_t flags, vrprpd_instance** out);

void vrprpd_instance_destroy(vrprpd_instance* inst);

/* Copy the instance's (n+1)^2 distance matrix into host memory d_host. */
int vrprpd_instance_get_dist(const vrprpd_instance* inst, int32_t* d_host);

/* A batch of candidates of one instance.
 *   ops  num x 2n int32, candidate i at ops + i*2n (4-byte aligned).
 *   off  num x (m+1) int32, candidate i at off + i*(m+1). */
typedef struct {
    int32_t num;
    const int32_t* ops;
    const int32_t* off;
} vrprpd_batch;

/*
 * Evaluate a batch (Section 3.1 Eqs. 7-23; the repair's "two-pass timing
 * evaluation", Section 4.2.3, done exactly): for each candidate, drop times,
 * pickup waits across vehicles, capacity and pool checks, makespan.
 *   makespan  num int32: the makespan, or INT32_MAX for CYCLE/MALFORMED.
 *   status    num uint32: VRPRPD_* bits.
 * Asynchronous on stream.  Device pointers.  One persistent launch over the
 * whole batch: each warp reads a tile of candidates with coalesced loads into
 * shared memory (as 16-bit codes) and walks all their routes in lock step.
 * Needs m <= 32, 2n+1 < 4096 and max d < 2^19 (VRPRPD_EINVAL otherwise; the
 * plain form below has no such limit).
 */
int vrprpd_evaluate(const vrprpd_instance* inst, const vrprpd_batch* batch, int32_t* makespan,
                    uint32_t* status, void* stream);

/* Same result as vrprpd_evaluate from HOST buffers (ops/off/makespan/status
 * all host pointers), returning when done.  Pinned (page-locked) ops and off
 * are read by the kernel in place over the host link, always by the staged
 * walk (its coalesced reads; the best staged shape vrprpd_autotune saw);
 * pageable ones are copied to the device first.  Results are copied back. */
int vrprpd_evaluate_host(const vrprpd_instance* inst, const vrprpd_batch* host_batch,
                         int32_t* makespan_host, uint32_t* status_host, void* stream);

/* A batch with 16-bit op codes and offsets: the same values as vrprpd_batch
 * in half the bytes (every op code of an instance the batched form accepts
 * is below 4096, so nothing is lost).
 *   ops  num x 2n uint16, candidate i at ops + i*2n (base 4-byte aligned).
 *   off  num x (m+1) uint16, candidate i at off + i*(m+1) (2-byte aligned). */
typedef struct {
    int32_t num;
    const uint16_t* ops;
    const uint16_t* off;
} vrprpd_batch16;

/* vrprpd_evaluate on a 16-bit batch (the same evaluation of Section 3.1,
 * Eqs. 7-23): same results (a code or offset out of range is MALFORMED as
 * before), same arguments, limits, errors and stream semantics, device
 * pointers.  Halves the candidate bytes each evaluation reads. */
int vrprpd_evaluate16(const vrprpd_instance* inst, const vrprpd_batch16* batch, int32_t* makespan,
                      uint32_t* status, void* stream);

/* vrprpd_evaluate_host on a 16-bit batch (host pointers; pinned buffers are
 * read in place, pageable ones copied first; returns when done).  Halves the
 * bytes that cross the host link. */
int vrprpd_evaluate16_host(const vrprpd_instance* inst, const vrprpd_batch16* host_batch,
                           int32_t* makespan_host, uint32_t* status_host, void* stream);

/* The plain GPU form kept as the comparison baseline: one thread per
 * candidate, distances read from global memory, no shared-memory staging,
 * no tuning.  Same results.  Allocates its per-thread scratch (ready times,
 * route cursors) on the first call and reuses it. */
int vrprpd_evaluate_plain(const vrprpd_instance* inst, const vrprpd_batch* batch,
                          int32_t* makespan, uint32_t* status, void* stream);

/*
 * vrprpd_evaluate_plain without any device allocation.  The paper has no
 * counterpart; this exists for callers that cannot let a library allocate
 * device memory: code recording a CUDA graph, serving processes that reserve
 * their memory budget up front, and processes whose framework caching
 * allocator already holds the free memory.
 *   Same arguments, results and stream semantics as vrprpd_evaluate_plain.
 *   Scratch: a fixed 16 MiB array inside the library image (4 Mi int32 words),
 *   present on every GPU that loads the library until the process exits.  A
 *   call needs (n+1) + 3m + ceil((2n+2)/32) words per thread and fails with
 *   VRPRPD_EINVAL when that leaves room for fewer than 32 threads (n above
 *   about 123 000 at small m).  The launch never has more threads than the
 *   scratch holds: blocks of up to 128 threads (a multiple of 32, fewer when
 *   fewer fit), and no more blocks than fit (vrprpd_evaluate_plain_noalloc_shape
 *   below gives the shape).
 *   Every call looks up the array's address on the current device (a runtime
 *   query, not an allocation), so the entry point stays valid across
 *   cudaDeviceReset.  The first call on a device may load the library's
 *   device code there; make it before any stream capture.  Every call shares
 *   the one array: calls whose kernels overlap on the GPU (different streams,
 *   or host threads without ordering) race on it.  The kernel initialises
 *   every scratch word it reads, so leftover contents from a previous call
 *   are harmless.
 */
int vrprpd_evaluate_plain_noalloc(const vrprpd_instance* inst, const vrprpd_batch* batch,
                                  int32_t* makespan, uint32_t* status, void* stream);

/* The launch shape vrprpd_evaluate_plain_noalloc uses for num candidates of an
 * instance with n customers and m vehicles: *blocks blocks of *threads
 * threads, with blocks x threads never above what the fixed scratch holds.
 * Host only (no CUDA call); VRPRPD_EINVAL when fewer than 32 threads fit or
 * an argument is out of range (n >= 1, m >= 1, num >= 0). */
int vrprpd_evaluate_plain_noalloc_shape(int32_t n, int32_t m, int64_t num, int32_t* blocks,
                                        int32_t* threads);

/*
 * Coordination counts of Section 5.2 ("Key Metrics"; the paper reports them
 * as percentages of n) for a batch of complete solutions:
 *   cross        num int32: customers whose dropoff and pickup are made by
 *                different vehicles (Cross-Agent);
 *   interleaved  num int32: customers whose dropoff vehicle does something
 *                else between their dropoff and pickup (Interleaved).  On one
 *                vehicle: the pickup does not directly follow the dropoff in
 *                the route.  On two vehicles: the dropoff vehicle has a next
 *                op and reaches it (dropoff time plus travel) strictly before
 *                the pickup completes (max(arrival, T_drop + p), Eqs. 8-10).
 * -1 marks an undefined count: both for a malformed candidate (an op code out
 * of range or repeated, offsets not 0 <= ... <= 2n), interleaved for a
 * precedence cycle.  Needs m <= 32 and (2n+1) max d + n max p < 2^31
 * (VRPRPD_EINVAL otherwise).  Device pointers; asynchronous on stream.
 */
int vrprpd_coordination(const vrprpd_instance* inst, const vrprpd_batch* batch, int32_t* cross,
                        int32_t* interleaved, void* stream);

/* Wait for stream and report a device-side error the kernels recorded for
 * this instance (VRPRPD_ETIMEOUT if a bounded wait gave up), then clear it. */
int vrprpd_sync(const vrprpd_instance* inst, void* stream);

/* Shape of the batched evaluation kernel: candidates per warp, warps per
 * block and how distances are read.  Set by vrprpd_autotune or by hand. */
#define VRPRPD_DIST_AUTO 0
#define VRPRPD_DIST_SMEM32 1   /* whole int32 matrix in shared memory */
#define VRPRPD_DIST_SMEM16 2   /* whole uint16 matrix in shared memory */
#define VRPRPD_DIST_GLOBAL16 3 /* uint16 matrix gathered from L2 */
#define VRPRPD_DIST_GLOBAL32 4 /* int32 matrix gathered from L2 */
#define VRPRPD_DIST_COORDS 5   /* recomputed exactly from coordinates in shared memory */
/* How a warp walks its candidates:
 *   VRPRPD_WALK_STAGED    each warp reads a tile of floor(32/m) candidates
 *                         with coalesced loads, checks every code (range,
 *                         duplicates) and keeps them as 16-bit codes in shared
 *                         memory, then walks them there;
 *   VRPRPD_WALK_STREAMED  each route's lane reads its own codes from global
 *                         memory through a register queue while it walks and
 *                         checks them on the way (a blocked walk gets the full
 *                         check afterwards); a group of group_warps warps (1
 *                         or 2) walks floor(32 group_warps / m) candidates, so
 *                         for m = 20 two warps walk three candidates.  Shared
 *                         memory holds only the ready times and offsets. */
#define VRPRPD_WALK_STAGED 0
#define VRPRPD_WALK_STREAMED 1
typedef struct {
    int32_t dist_mode;
    int32_t warps_per_block;
    int32_t blocks_per_sm;     /* 0 = as many as fit */
    int32_t walk;              /* VRPRPD_WALK_STAGED or VRPRPD_WALK_STREAMED */
    int32_t group_warps;       /* streamed walk: warps per candidate group (1 or 2) */
} vrprpd_eval_config;

int vrprpd_eval_set_config(vrprpd_instance* inst, const vrprpd_eval_config* cfg);
int vrprpd_eval_get_config(const vrprpd_instance* inst, vrprpd_eval_config* cfg);
/* Time each feasible configuration on `batch` (device) and keep the fastest.
 * The choice holds for batches like the one timed: give it at least a few
 * tiles (floor(32/m) candidates each) per warp of a full GPU, or it favours
 * shapes that only suit a batch too small to fill the SMs. */
int vrprpd_autotune(vrprpd_instance* inst, const vrprpd_batch* batch, void* stream,
                    vrprpd_eval_config* chosen);

/* ---- many instances of uneven size in one persistent launch ---- */
typedef struct vrprpd_multi vrprpd_multi;

/* Plan one persistent launch over n_inst (instance, batch) pairs (Section
 * 4.2.1's multi-instance parallelism applied to evaluation): the tiles of all
 * batches form one work list; every warp takes tiles in turn, whatever
 * instance they belong to.  insts, batches, makespan and status are HOST
 * arrays of n_inst entries; the batch and output pointers they hold are
 * DEVICE pointers that must stay valid while the plan is used.  All instances
 * must live on one device and satisfy the batched evaluator's limits. */
int vrprpd_multi_create(const vrprpd_instance* const* insts, const vrprpd_batch* batches,
                        int32_t* const* makespan, uint32_t* const* status, int32_t n_inst,
                        vrprpd_multi** out);
/* Evaluate every batch of the plan, asynchronously on stream.  On a non-NULL
 * stream that is not being captured the first call captures the launch as a
 * CUDA graph and later calls replay it; inside a caller's capture (or on the
 * NULL stream) it launches directly.  Results as vrprpd_evaluate. */
int vrprpd_multi_evaluate(vrprpd_multi* plan, void* stream);
/* Time the walk (staged, or streamed with one-warp groups), warps per block
 * and distance mode (GLOBAL16/GLOBAL32) on the plan's own batches; keep the
 * fastest. */
int vrprpd_multi_autotune(vrprpd_multi* plan, void* stream, vrprpd_eval_config* chosen);
/* Set the plan's shape by hand: dist_mode GLOBAL16 (every instance with a
 * 16-bit matrix) or GLOBAL32, warps_per_block 1..32, walk staged or streamed
 * with group_warps 1 (Section 4.2.1's multi-instance parallelism, the same
 * evaluation).  VRPRPD_EINVAL when the shape does not fit. */
int vrprpd_multi_set_config(vrprpd_multi* plan, const vrprpd_eval_config* cfg);
void vrprpd_multi_destroy(vrprpd_multi* plan);

/* ======================================================================== */
/* ALNS (Section 4.2, Algorithm 1) on the device                             */
/* ======================================================================== */

/* A solution in HOST memory: ops[2n] and off[m+1] (caller-owned). */
typedef struct {
    int32_t* ops;
    int32_t* off;
    int32_t makespan;
    uint32_t status;
} vrprpd_solution;

/* Hyperparameters (Table 2).  vrprpd_alns_params_default() fills the paper's
 * values: T0 = 0.30, alpha = 0.9998, reheat 0.50, stagnation 2000, tau = 100,
 * r = 0.1, sigma = (33, 9, 13), minimum weight 0.1, q from Section 4.2.2. */
typedef struct {
    double T0, alpha, reheat, r;
    int32_t stagnation, tau;
    int32_t sigma1, sigma2, sigma3;
    double w_min;
    int32_t q_min, q_max;      /* 0, 0 = q_max = max(4, floor(0.05 n)), q_min = max(4, floor(q_max/2)) */
    int32_t iterations;
    int32_t repair_mask;       /* bit 0 greedy, bit 1 regret-2, bit 2 regret-3, bit 3 regret-m insertion
                                  (Section 4.2.3; default 3).  Regret-k: options are the best insertion
                                  per dropoff vehicle; regret = sum over the k best of (c_i - c_1),
                                  a missing option counting 2^40 */
    int32_t team_blocks;       /* CTAs cooperating on one instance; 0 = chosen from n */
    int32_t destroy_mask;      /* Section 4.2.2 destroy operators (default 1):
                                  bit 0 random: q customers by partial Fisher-Yates;
                                  bit 1 worst: removal gains z(S) - z(S - c), ranked largest first, q
                                    roulette draws with weight r^-6 on the r-th remaining;
                                  bit 2 Shaw: a random seed and the q-1 customers most related to it,
                                    i.e. smallest 18 d + 6 |T_drop diff| + 5 [drop vehicles differ] +
                                    5 [pickup vehicles differ] (2R with phi 9, chi 3, omega 5);
                                  bit 3 cluster: a random centre and its q-1 nearest by travel time;
                                  bit 4 route: a random non-empty route's customers, topped up to q_min
                                    by the least travel time from a removed customer (with this bit on,
                                    up to n customers await reinsertion, so the run's per-customer
                                    device buffers take n rows instead of q_max);
                                  bit 5 critical path: q random customers of the latest-returning route
                                    (all if fewer), topped up to q_min by the latest pickup completion.
                                  Ties go to the smaller customer id. */
    int32_t ls_pickup_every;   /* Section 4.2.6 periodic local search on the current solution, after the
                                  acceptance step of every k-th iteration (0 = off).  Pickup
                                  repositioning (default 200): customers whose pickup is on a vehicle
                                  returning at 95% of the makespan or later may move that pickup to any
                                  position of any vehicle.  Cross-agent relocation (ls_relocate_every,
                                  default 500): customers with an op on the bottleneck vehicle (latest
                                  return, lower index on ties) may move both ops onto one other vehicle.
                                  Each pass applies the move with the least (makespan, travel, customer,
                                  flat gap index) if it lowers the makespan; up to three passes;
                                  pickup repositioning first when both fall due. */
    int32_t ls_relocate_every;
    int32_t replicas;          /* Section 4.2.1 multi-instance parallelism: independent ALNS instances of
                                  this one problem in one launch (default 1, 0 reads as 1; the paper
                                  runs 32 per GPU),
                                  each a team of CTAs with its own solution, temperature, weights and
                                  draw stream (replica 0 draws like a single run).  The resident CTAs
                                  of the GPU are shared among them. */
    int32_t sync_every;        /* every sync_every-th iteration (default 1000; 0 = never) all replicas
                                  meet, and each whose best is worse than the best of all (lowest
                                  index among equal bests) takes that solution as its current and best.
                                  The paper's replicas poll without meeting; meeting makes runs
                                  reproducible. */
    int32_t init_mode;         /* start solution when init is NULL: 1 (default) the paper's
                                  vrprpd_initial_solution_paper, 0 the plain sweep of
                                  vrprpd_initial_solution */
    int32_t init_refine_rounds;/* refinement rounds of that start (default 10; 0 = the constructor alone) */
    int64_t wait_limit_ns;     /* limit of each device-side wait of the team (its barriers), in ns: a
                                  wait that runs out ends the run with VRPRPD_ETIMEOUT instead of
                                  hanging (default 2 s; 0 = the default) */
} vrprpd_alns_params;

typedef struct {
    int32_t iterations, accepted, improved, new_best, reheats, rejected_infeasible;
    int32_t z_init, z_best, z_current;
    double T_final;
    double w_destroy[8], w_repair[4];  /* final operator weights (destroy 0-5 used) */
    double device_ms;          /* wall time of the device run */
    int64_t matrix_entries;    /* insertion-matrix entries scored by the O(1) tile formula */
    int64_t fallback_entries;  /* entries with a shortcut gap: exact from simulations with one stop
                                  (both gaps shortcuts: both stops) instead of the tile formula */
    int32_t team_blocks;       /* CTAs used */
    double phase_ms[6];        /* wall time per phase: begin, prep, gaps, matrix, select, end */
    int64_t incremental_steps; /* greedy steps whose longest-path table was updated in O(N^2) */
    int64_t full_steps;        /* greedy steps that re-walked W from every op (after a removal or a
                                  shortcut insertion) */
    int32_t ls_moves;          /* local-search moves applied */
    int32_t ls_new_best;       /* iterations whose local search gave a new best solution */
    double ls_ms;              /* wall time spent in the local search */
    int32_t replicas;          /* replicas run; the counters above are summed over them, z_current,
                                  T_final, the weights and phase times are replica 0's */
    int32_t imports;           /* best-of-all solutions taken at checkpoints, over all replicas */
    int32_t best_replica;      /* the replica whose best solution is returned */
    int64_t pruned_entries;    /* of matrix_entries, those never scored: a lower bound over their
                                  tile showed that none of them can be the one the repair operator
                                  picks (its per-vehicle bests, or the best, are already at or
                                  below it); the result is the same as scoring them */
    int64_t tiles;             /* insertion-matrix tiles (32 drop gaps x 64 pickup gaps) run */
    int64_t tiles_pruned;      /* of those, tiles in which no customer was left to score */
} vrprpd_alns_stats;

void vrprpd_alns_params_default(vrprpd_alns_params* params);

/* Deterministic feasible start (host): customers in exact angular order
 * around the depot (by id when the instance has no coordinates), split into
 * m sectors of balanced workload w_c = 2 d(0,c) + p_c, each route serving its
 * sector in blocks "D c1..cb, P c1..cb" with b = min(Q, R / min(m, R)).
 * out->ops / out->off are host buffers of 2n and m+1 int32; needs R, Q >= 1. */
int vrprpd_initial_solution(const vrprpd_instance* inst, vrprpd_solution* out);

/*
 * The paper's three-phase initial solution (Section 4.2.5), built on the
 * device, then refined:
 *   1. customers by exact angle around the depot (by id for an instance made
 *      from a distance matrix), cut into m' = min(m, R) sectors of equal count;
 *   2. load balancing on w_c = 2 d(0,c) + p_c: while the spread of the sector
 *      workloads is at least 10% of their mean, the heaviest sector (lowest
 *      index on ties) hands its boundary customer to its lighter neighbour,
 *      as long as that lowers the heavier of the two (at most 4n moves);
 *   3. nearest-neighbour routes: vehicle v serves sector v alone, leaving the
 *      depot with b = min(Q, floor(R/m')) resources, each step taking the
 *      feasible op that completes first (ties: travel, drop before pickup,
 *      op code).
 * Refinement: up to refine_rounds rounds of the periodic local search
 * (pickup repositioning, then cross-agent relocation, three passes each),
 * stopping at the first round that moves nothing.
 *   out  host buffers (2n ops, m+1 offsets); out->makespan is set.
 * Needs what vrprpd_alns_run needs.  Blocking: returns when done.
 */
int vrprpd_initial_solution_paper(const vrprpd_instance* inst, int32_t refine_rounds, vrprpd_solution* out,
                                  void* stream);

/*
 * Run Algorithm 1 on the device: roulette selection of the enabled destroy
 * and repair operators (Sections 4.2.2-4.2.3) over the full insertion-delta
 * matrix, simulated-annealing acceptance with the text's reheat gate, adaptive
 * weights, the periodic local search (Section 4.2.6) and, with several
 * replicas, the multi-instance checkpoints (Section 4.2.1).  Every random draw
 * is SplitMix64 of (seed-derived key, iteration-derived counter), so a run is
 * reproducible bit for bit.
 *   init     host solution to start from, or NULL for vrprpd_initial_solution.
 *            It must be feasible (status 0).
 *   best     host buffers receive the best solution found (and its makespan),
 *            over all replicas.
 *   current  host buffers for replica 0's final current solution, or NULL.
 *   stats    may be NULL; z_trace (host, replicas x params->iterations int32,
 *            replica-major) receives each replica's current makespan after
 *            each iteration, or NULL.
 * Needs m <= 32, 2n + m <= 4096, max d < 2^17 and (2n+1)*max(d) + n*max(p) < 2^27
 * (VRPRPD_EINVAL otherwise).  Blocking: returns when done.
 */
int vrprpd_alns_run(const vrprpd_instance* inst, const vrprpd_solution* init,
                    const vrprpd_alns_params* params, uint64_t seed, vrprpd_solution* best,
                    vrprpd_solution* current, vrprpd_alns_stats* stats, int32_t* z_trace, void* stream);

/*
 * The insertion-delta matrix of Section 4.2.3 for one customer c (absent from
 * the partial solution given in host memory: ops[off[m]], off[m+1]).  Rows are
 * the dropoff gaps, columns the pickup gaps, gaps enumerated route by route
 * (route v has off[v+1]-off[v]+1 gaps).  delta_host (G x G, G = off[m] + m)
 * receives z(S + D_c + P_c) - z(S), or INT32_MAX when that solution has a
 * precedence cycle, breaks capacity on a receiving vehicle or the pool;
 * travel_host (G x G, may be NULL) receives the change in total route length.
 * Computed by the same kernels the ALNS uses.  Blocking.
 */
int vrprpd_insertion_matrix(const vrprpd_instance* inst, const int32_t* ops_host,
                            const int32_t* off_host, int32_t c, int32_t* delta_host,
                            int32_t* travel_host, void* stream);

/*
 * The repair of Section 4.2.3 stopped part way, for checking its later
 * steps: the partial solution (host ops[off[m]], off[m+1], holding every
 * customer but the `count` ascending ids in `removed`) is repaired for
 * `steps` insertions (0 <= steps < count) by repair operator repair_op (0
 * greedy, 1 regret-2, 2 regret-3, 3 regret-m) exactly as an ALNS iteration
 * does, on a team of team_blocks CTAs (0 = the whole GPU): after an insertion
 * whose two gaps are no shortcuts the next step updates the longest-path
 * table in place instead of re-walking the solution.  Then the insertion
 * matrix of the first customer still to insert (the smallest remaining id) is
 * written out as vrprpd_insertion_matrix writes it.
 *   out_ops/out_off  host, off[m] + 2 steps ops and m + 1 offsets: the
 *                    partial solution after the steps.
 *   delta/travel     host, G x G with G = off[m] + 2 steps + m (travel may be NULL).
 *   incremental_steps  host, may be NULL: steps (the dump's included) whose
 *                    table was updated in place.
 * VRPRPD_EINVAL if a customer has no feasible insertion on the way.  Blocking.
 */
int vrprpd_repair_then_matrix(const vrprpd_instance* inst, const int32_t* ops_host, const int32_t* off_host,
                              const int32_t* removed_host, int32_t count, int32_t repair_op, int32_t steps,
                              int32_t team_blocks, int32_t* out_ops_host, int32_t* out_off_host,
                              int32_t* delta_host, int32_t* travel_host, int64_t* incremental_steps,
                              void* stream);

/* ======================================================================== */
/* BRKGA (Section 4.4, Algorithm 2) on the device                            */
/* ======================================================================== */

/* Chromosome layouts, float32 keys in [0,1).  Both start with the 2n op
 * priorities: keys[2(c-1)+isPickup] for customer c's dropoff/pickup (lower =
 * scheduled first, Section 4.4.1).
 *   VRPRPD_LAYOUT_VKEYS (L = 2n + m): keys[2n+v] orders the vehicles for
 *     SelectVehicle's tie-break (lower key = preferred).
 *   VRPRPD_LAYOUT_HINTS (L = 4n, the paper's (pi, alpha)): keys[2n + o-2] is
 *     op o's assignment hint alpha_o; among the vehicles at the least arrival
 *     op o goes to h = floor(m * alpha_o) (fp64, capped at m-1), else to the
 *     next one in cyclic order h+1, h+2, ... (mod m). */
#define VRPRPD_LAYOUT_VKEYS 0
#define VRPRPD_LAYOUT_HINTS 1

typedef struct {
    int32_t pop, generations;
    int32_t warm_slots;        /* slots seeded from the warm start (0 without one);
                                  negative: ceil(0.15 pop), Section 4.4.4 */
    int32_t warm_variants;     /* distinct warm variants cycled over those slots (20) */
    float elite_frac, mutant_frac, rho;  /* Table 3: 0.15, 0.15, 0.7 */
    float eps;                 /* warm perturbation half-width (0.03, Section 4.4.4) */
    int32_t layout;            /* VRPRPD_LAYOUT_VKEYS (default) or VRPRPD_LAYOUT_HINTS */
} vrprpd_brkga_params;

/* Table 3 values: pop 30000, 20000 generations, elite/mutant 0.15, rho 0.7,
 * warm slots -1 (= ceil(0.15 pop)), 20 variants, eps 0.03; layout VRPRPD_LAYOUT_VKEYS. */
void vrprpd_brkga_params_default(vrprpd_brkga_params* params);

/*
 * Decode a batch of chromosomes (Algorithm 2): stable argsort of the 2n
 * priorities (ties by op index), then passes over the ops in that order; a
 * dropoff is feasible on a vehicle that can load one more resource within Q
 * and the pool R; a pickup is feasible once its dropoff is scheduled, on a
 * vehicle with room; SelectVehicle takes the least arrival time t[v] +
 * d(l[v], c), ties by the layout's rule (vehicle keys or the op's hint); the
 * pickup leaves at max(arrival, T_drop + p_c).  Passes stop when everything
 * is scheduled or a pass schedules nothing.
 *   keys     device, num x L float32 (L by layout: 2n + m or 4n).
 *   layout   VRPRPD_LAYOUT_VKEYS or VRPRPD_LAYOUT_HINTS (else VRPRPD_EINVAL).
 *   ops/off  device, num x 2n and num x (m+1): the decoded routes (scheduled ops only).
 *   z        device, num: makespan of the decoded routes.
 *   unsched  device, num: ops left unscheduled.
 *   fitness  device, num int64: z + 10^6 * unsched (Section 4.4.2, infeasibility handling).
 * Asynchronous on stream.  Needs m <= 32 and 2n + m <= 8192.
 */
int vrprpd_brkga_decode(const vrprpd_instance* inst, const float* keys, int32_t num, int32_t layout,
                        int32_t* ops, int32_t* off, int32_t* z, int32_t* unsched, int64_t* fitness,
                        void* stream);

/*
 * Run the BRKGA: warm-started population (slot 0 = the exact encoding of
 * `warm`, pi_o = (r-1)/L_v and vehicle key v/m, or every op's hint v/m rounded
 * up so that floor(m * alpha) = v under VRPRPD_LAYOUT_HINTS; slots 1..warm_slots-1 cycle
 * through perturbed variants, key + U(-eps, eps) clamped to [0, 1-2^-24];
 * the rest uniform random), then per generation: decode, re-evaluate the
 * decoded routes with the batched evaluator, rank by (fitness, index), copy
 * the elites, draw mutants, and fill the rest by biased crossover (elite gene
 * with probability rho).  One generation is a CUDA graph replayed
 * `generations` times.
 *   warm          host solution or NULL (random start).
 *   best          host buffers: routes of the best chromosome of the last generation.
 *   best_fitness  host, may be NULL.
 *   trace         host, `generations` int64 (best fitness per generation) or NULL.
 *   final_keys    device, pop x L float32 (the last population) or NULL.
 * Needs pop <= 16384, m <= 32 and 2n + m <= 8192.  Blocking.
 */
int vrprpd_brkga_run(const vrprpd_instance* inst, const vrprpd_brkga_params* params,
                     const vrprpd_solution* warm, uint64_t seed, vrprpd_solution* best,
                     int64_t* best_fitness, int64_t* trace, float* final_keys, void* stream);

/* ======================================================================== */
/* Serving: continuous batching of solve requests                            */
/* ======================================================================== */

/* A solve request: the instance (host arrays, copied at submit) and the
 * pipeline's budgets.  The server runs ALNS from the deterministic start
 * solution, then BRKGA warm-started from the ALNS incumbent (Section 4,
 * "sequential two-stage pipeline"), and answers with the better of the two. */
typedef struct {
    const int32_t* coords;     /* host, (n+1) x 2 */
    const int32_t* p;          /* host, n */
    int32_t n, m, R, Q;
    uint32_t flags;
    vrprpd_alns_params alns;   /* iterations >= 1; team_blocks is set by the server */
    vrprpd_brkga_params brkga; /* generations = 0 skips BRKGA */
    uint64_t seed;
} vrprpd_request;

typedef struct {
    int64_t id;
    int32_t status;            /* VRPRPD_OK or the error the request hit */
    int32_t z_alns, z_brkga, z_best;
    double t_submit_ms, t_start_ms, t_end_ms;   /* server clock */
    double device_ms;
    int32_t n, m;
    char message[160];         /* error text when status != VRPRPD_OK */
} vrprpd_result;

typedef struct {
    int32_t submitted, completed, pending, active, peak_active;
    size_t bytes_in_use, peak_bytes;
    double p50_ms, p99_ms;     /* submit-to-finish latency of completed requests */
} vrprpd_server_stats;

typedef struct vrprpd_server vrprpd_server;

/* Start a server on the current device with max_active worker slots.  A
 * request is admitted (FIFO) when a slot is free, its estimated device memory
 * fits what mem_budget leaves, and its ALNS team fits the resident-CTA share;
 * admitted requests run concurrently on their own streams.  Results do not
 * depend on what else runs: every draw is counter-based. */
int vrprpd_server_create(size_t mem_budget, int32_t max_active, vrprpd_server** out);
/* Queue a request; VRPRPD_EBUSY if it alone exceeds the memory budget. */
int vrprpd_server_submit(vrprpd_server* server, const vrprpd_request* req, int64_t* id);
/* VRPRPD_ENOTREADY until the request finished; then fills *out and, when the
 * host buffers are given, the best routes (ops[2n], off[m+1]). */
int vrprpd_server_poll(vrprpd_server* server, int64_t id, vrprpd_result* out, int32_t* ops, int32_t* off);
/* Blocking form of poll. */
int vrprpd_server_wait(vrprpd_server* server, int64_t id, vrprpd_result* out, int32_t* ops, int32_t* off);
int vrprpd_server_get_stats(vrprpd_server* server, vrprpd_server_stats* out);
/* Withdraw every request still waiting for admission (requests already
 * running finish).  Each withdrawn request completes at once with status
 * VRPRPD_EBUSY and the message "withdrawn before admission"; *withdrawn (may
 * be NULL) receives their count.  Serves a bounded serving window. */
int vrprpd_server_cancel_pending(vrprpd_server* server, int32_t* withdrawn);
/* Finish everything queued, stop the workers, free the server. */
void vrprpd_server_destroy(vrprpd_server* server);

const char* vrprpd_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
