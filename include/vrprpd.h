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
 * whole batch: each warp stages a tile of candidates in shared memory with a
 * TMA bulk copy and walks all their routes in lock step.
 */
int vrprpd_evaluate(const vrprpd_instance* inst, const vrprpd_batch* batch, int32_t* makespan,
                    uint32_t* status, void* stream);

/* Same result as vrprpd_evaluate from HOST buffers (ops/off/makespan/status
 * all host pointers): copies in, evaluates, copies out, returns when done. */
int vrprpd_evaluate_host(const vrprpd_instance* inst, const vrprpd_batch* host_batch,
                         int32_t* makespan_host, uint32_t* status_host, void* stream);

/* The plain GPU form kept as the comparison baseline: one thread per
 * candidate, distances read from global memory, no shared-memory staging,
 * no tuning.  Same results.  Allocates its per-thread scratch (ready times,
 * route cursors) on the first call and reuses it. */
int vrprpd_evaluate_plain(const vrprpd_instance* inst, const vrprpd_batch* batch,
                          int32_t* makespan, uint32_t* status, void* stream);

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
typedef struct {
    int32_t dist_mode;
    int32_t warps_per_block;
    int32_t blocks_per_sm;     /* 0 = as many as fit */
} vrprpd_eval_config;

int vrprpd_eval_set_config(vrprpd_instance* inst, const vrprpd_eval_config* cfg);
int vrprpd_eval_get_config(const vrprpd_instance* inst, vrprpd_eval_config* cfg);
/* Time each feasible configuration on `batch` (device) and keep the fastest. */
int vrprpd_autotune(vrprpd_instance* inst, const vrprpd_batch* batch, void* stream,
                    vrprpd_eval_config* chosen);

const char* vrprpd_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
