/*
 * VRP-RPD CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously-correct C written from the paper's problem statement
 * (Section 3.1, Eqs. 1-22) and algorithms (Algorithm 1, Algorithm 2, Section
 * 4.2-4.4).  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load this library; the product library never links or calls it.
 * It shares no code, header or table with the CUDA library.
 *
 * Conventions: customers 1..n, depot 0, op code o = 2c + isPickup.
 * A candidate is route-major: ops[off[v] .. off[v+1]) is vehicle v's sequence.
 * Status bits: 1 CYCLE, 2 VEH_CAP, 4 POOL, 8 MALFORMED.
 */
#ifndef VRPRPD_ORACLE_H
#define VRPRPD_ORACLE_H
#include <stdint.h>

#define OR_CYCLE 1u
#define OR_VEH_CAP 2u
#define OR_POOL 4u
#define OR_MALFORMED 8u
#define OR_LOAD_FULL 1u

typedef struct {
    int32_t n, m, R, Q;
    uint32_t flags;      /* OR_LOAD_FULL or 0 (minimal load, the default) */
    const int32_t* d;    /* (n+1)*(n+1) travel times, row-major */
    const int32_t* p;    /* n processing times, p[c-1] for customer c */
} oracle_inst;

/* EUC_2D (TSPLIB): d(i,j) = nint(sqrt(dx^2+dy^2)), computed in double. */
void oracle_euc2d(const int32_t* coords, int32_t n_nodes, int32_t* d);

/* Evaluate one candidate.  allow_partial=1 accepts a subset of customers
 * (each present customer with both ops), total ops = off[m].
 * Returns 0, or -1 if a time exceeds INT32_MAX (never for valid instances).
 * times (optional, size 2n+2 indexed by op code) receives each op's
 * departure time (drop: arrival) or INT64_MIN if unprocessed. */
int oracle_evaluate(const oracle_inst* I, const int32_t* ops, const int32_t* off,
                    int allow_partial, int32_t* z, uint32_t* status, int64_t* times);

/* Section 5.2 coordination counts (cross-agent, interleaved) of one complete
 * solution; -1 where undefined.  Returns the evaluator's status bits. */
uint32_t oracle_coordination(const oracle_inst* I, const int32_t* ops, const int32_t* off, int32_t* cross,
                             int32_t* interleaved);
void oracle_evaluate_batch(const oracle_inst* I, int32_t count, const int32_t* ops,
                           const int32_t* off, int32_t* z, uint32_t* status, int32_t threads);

/* Shortest-path closure of d (Floyd-Warshall), for lower-bound invariants. */
void oracle_sp_closure(const int32_t* d, int32_t n_nodes, int64_t* sp);

/* Exhaustive optimum over all candidates (every op order, every split into m
 * routes); returns the best makespan among status==0 candidates, or -1. */
int64_t oracle_bruteforce(const oracle_inst* I, int32_t* best_ops, int32_t* best_off);

/* Min-max VRP optimum by enumeration of customer orders and splits (each
 * customer visited once, route length = travel only). */
int64_t oracle_minmax_vrp(const int32_t* d, int32_t n, int32_t m);

/* Held-Karp TSP tour length over nodes 0..n. */
int64_t oracle_held_karp(const int32_t* d, int32_t n);

/* ---- counter-based RNG and exp (independent restatements) ---- */
uint64_t oracle_splitmix64_next(uint64_t* state);
uint64_t oracle_rng(uint64_t key, uint64_t counter);
double oracle_exp(double x);

/* ---- ALNS (Algorithm 1) ---- */
typedef struct {
    double T0, alpha, reheat, r;          /* 0.30, 0.9998, 0.50, 0.1 */
    int32_t stagnation, tau;              /* 2000, 100 */
    int32_t sigma1, sigma2, sigma3;       /* 33, 9, 13 */
    double w_min;                         /* 0.1 */
    int32_t q_min, q_max;                 /* 0 = paper formula */
    int32_t iterations;
    int32_t repair_mask;                  /* bit0 greedy, bit1 regret-2, bit2 regret-3, bit3 regret-m */
    int32_t destroy_mask;                 /* bit0 random, 1 worst, 2 Shaw, 3 cluster, 4 route, 5 critical path */
    int32_t ls_pickup_every;              /* pickup repositioning period (200; 0 = off) */
    int32_t ls_relocate_every;            /* cross-agent relocation period (500; 0 = off) */
} oracle_alns_params;

typedef struct {
    int32_t iterations, accepted, improved, new_best, reheats, rejected_infeasible;
    int32_t z_init, z_best, z_current;
    double T_final;
    double w_destroy[8], w_repair[4];
    int32_t ls_moves, ls_new_best;        /* local-search moves applied; best solutions it found */
} oracle_alns_stats;

void oracle_q_range(int32_t n, int32_t* q_min, int32_t* q_max);

/* Insertion-delta matrix for customer c into partial solution (ops, off).
 * out has (N+m)^2 int32 entries, row = D gap, col = P gap (gaps enumerated
 * route by route, gap i of route v sits before the v-th route's op i).
 * Each entry = z(S') - z(S), or INT32_MAX when S' has any status bit.
 * Also writes the travel delta per entry (travel_out, may be NULL). */
int oracle_insertion_matrix(const oracle_inst* I, const int32_t* ops, const int32_t* off,
                            int32_t c, int32_t* out, int32_t* travel_out, uint32_t* status_out);

int oracle_initial_solution(const oracle_inst* I, const int32_t* coords, int32_t* ops, int32_t* off);

/* One destroy step (Section 4.2.2) on solution (S, So): operator di (0 random,
 * 1 worst, 2 Shaw, 3 cluster, 4 route, 5 critical path), removal size q,
 * top-up bound qmin, draws from (key, base + ...).  Marks rem[1..n]; returns
 * how many customers it removed. */
int oracle_destroy(const oracle_inst* I, int32_t di, const int32_t* S, const int32_t* So, int32_t q,
                   int32_t qmin, uint64_t key, uint64_t base, char* rem);

/* Periodic local search (Section 4.2.6) on a feasible complete solution, in
 * place: mode 1 pickup repositioning, mode 2 cross-agent relocation, up to
 * `passes` passes.  Returns the moves applied (z = the new makespan), or -1
 * on an infeasible input or a bad mode. */
int oracle_local_search(const oracle_inst* I, int32_t mode, int32_t passes, int32_t* ops, int32_t* off,
                        int32_t* z);

/* The repair operators alone (Section 4.2.3) on a partial solution (ops, off;
 * off[m] ops): reinsert the customers removed[0..count) (ascending ids), op
 * 0 greedy, 1 regret-2, 2 regret-3, 3 regret-m, one insertion per step, at
 * most max_steps steps (negative: all).  out_ops needs off[m] + 2 count
 * entries.  Returns 0, or -1 on bad arguments or when a customer has no
 * feasible insertion. */
int oracle_repair(const oracle_inst* I, int32_t op, const int32_t* ops, const int32_t* off, const int32_t* removed,
                  int32_t count, int32_t max_steps, int32_t* out_ops, int32_t* out_off);

/* Algorithm 1's acceptance and adaptation alone, on a scripted run: iteration
 * k (1-based) used destroy operator di[k-1] and repair operator rj[k-1], its
 * repaired candidate has makespan zn[k-1] and status st[k-1], and u[k-1] is
 * its SA draw.  Starts from makespan z0 (current = best), unit weights and
 * T = T0 z0, as oracle_alns_run does; fills stats (scores, weights, T,
 * counts) and z_trace (current makespan after each iteration). */
int oracle_alns_adapt_script(const oracle_alns_params* P, int32_t z0, int32_t iters, const int32_t* di,
                             const int32_t* rj, const int32_t* zn, const uint32_t* st, const double* u,
                             oracle_alns_stats* stats, int32_t* z_trace);

int oracle_alns_run(const oracle_inst* I, const int32_t* init_ops, const int32_t* init_off,
                    const oracle_alns_params* P, uint64_t seed,
                    int32_t* best_ops, int32_t* best_off, int32_t* cur_ops, int32_t* cur_off,
                    oracle_alns_stats* st, int32_t* z_trace);

/* R independent replicas of Algorithm 1 (Section 4.2.1, multi-instance
 * parallelism), replica r on its own draw stream (r = 0: the single-run
 * stream), all from the same start.  After every sync_every-th iteration each
 * replica whose best is worse than the best of all replicas (lowest index on
 * ties) takes it as its current and best solution.  stats and z_traces hold R
 * entries / R x iterations; best_* is the best of all. */
int oracle_alns_run_replicas(const oracle_inst* I, const int32_t* init_ops, const int32_t* init_off,
                             const oracle_alns_params* P, uint64_t seed, int32_t replicas, int32_t sync_every,
                             int32_t* best_ops, int32_t* best_off, int32_t* best_replica,
                             oracle_alns_stats* stats, int32_t* z_traces, int32_t* imports);

/* ---- BRKGA (Algorithm 2 decoder, Section 4.4) ---- */
/* Chromosome layouts.  Both start with 2n priority keys (op index
 * 2(c-1)+isPickup).  Layout 0 (2n+m keys): then m vehicle keys; SelectVehicle
 * ties go to the lower vehicle key.  Layout 1 (4n keys, Section 4.4.1): then
 * 2n assignment hints alpha_o; op o's ties go to the hinted vehicle
 * h = floor(m * alpha_o) (computed in fp64, at most m-1), then by increasing
 * cyclic distance (v - h) mod m. */
#define OR_LAYOUT_VKEYS 0
#define OR_LAYOUT_HINTS 1
int oracle_decode(const oracle_inst* I, const float* keys, int32_t* ops, int32_t* off,
                  int32_t* z, int32_t* unscheduled, int64_t* fitness);
int oracle_decode_l(const oracle_inst* I, const float* keys, int32_t layout, int32_t* ops, int32_t* off,
                    int32_t* z, int32_t* unscheduled, int64_t* fitness);

/* ALNS seed encoding (Section 4.4.4): pi_o = (r-1)/L_v; layout 0 vehicle
 * key v/m; layout 1 hint alpha_o = v/m for every op on vehicle v, rounded up
 * to the smallest float with m * alpha_o >= v, so that floor(m * alpha_o) = v. */
void oracle_encode(const oracle_inst* I, const int32_t* ops, const int32_t* off, float* keys);
void oracle_encode_l(const oracle_inst* I, const int32_t* ops, const int32_t* off, int32_t layout, float* keys);

/* The paper's three-phase initial solution (Section 4.2.5: sweep sectors,
 * load balancing below 10% imbalance, nearest-neighbour routes) and up to
 * refine_rounds rounds of its local-search refinement.  coords may be NULL. */
int oracle_initial_solution_paper(const oracle_inst* I, const int32_t* coords, int32_t refine_rounds,
                                  int32_t* ops, int32_t* off);

/* Construction seed h (0 nearest neighbour, 1 load-balanced, 2 shortest
 * processing time) of the BRKGA warm start as a chromosome (Section 4.4.4). */
void oracle_seed_chromosome(const oracle_inst* I, int32_t h, int32_t layout, float* keys);

typedef struct {
    int32_t pop, generations, warm_slots, warm_variants;
    float elite_frac, mutant_frac, rho;
    float eps;                            /* perturbation half-width, 0.03 */
    int32_t layout;                       /* OR_LAYOUT_VKEYS or OR_LAYOUT_HINTS */
} oracle_brkga_params;

int oracle_brkga_run(const oracle_inst* I, const oracle_brkga_params* P,
                     const int32_t* warm_ops, const int32_t* warm_off, uint64_t seed,
                     float* final_keys, int64_t* best_fitness_trace,
                     int32_t* best_ops, int32_t* best_off, int64_t* best_fitness);

#endif
