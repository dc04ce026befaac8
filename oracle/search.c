/*
 * VRP-RPD oracle: counter-based RNG, exp, ALNS (Algorithm 1) and BRKGA
 * (Section 4.4, Algorithm 2).  TEST INFRASTRUCTURE ONLY -- see oracle.h.
 *
 * Everything here is sequential and re-simulates from scratch: each entry of
 * an insertion-delta matrix is the evaluator run on the whole modified
 * solution.  Floating point is IEEE fp64/fp32 with no FMA contraction (the
 * library is compiled with -ffp-contract=off), so every rounding is the one
 * written in the source.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

/* ------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number     */
/* generators", OOPSLA 2014): state advances by the golden gamma, output is  */
/* the variant-13 finaliser of the state.  The counter form returns the      */
/* (counter+1)-th output of a generator seeded with key.                     */
/* ------------------------------------------------------------------------ */
static const uint64_t SM_GAMMA = 0x9E3779B97F4A7C15ull;

static uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t oracle_splitmix64_next(uint64_t* state) {
    *state += SM_GAMMA;
    return sm_mix(*state);
}

uint64_t oracle_rng(uint64_t key, uint64_t counter) { return sm_mix(key + (counter + 1) * SM_GAMMA); }

/* Stream keys: stream s of seed is the s-th draw of the seed itself. */
enum { STREAM_ALNS = 1, STREAM_BRKGA = 2, STREAM_WARM = 3 };
static uint64_t stream_key(uint64_t seed, uint64_t s) { return oracle_rng(seed, s); }

/* uniform integer in [0,k): high 32 bits scaled by k (multiply-shift) */
static int32_t rng_below(uint64_t r, int32_t k) { return (int32_t)(((r >> 32) * (uint64_t)k) >> 32); }
/* uniform double in [0,1) from 53 bits */
static double rng_unit(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }
/* float key in [0,1) from 24 bits */
static float rng_key(uint64_t r) { return (float)(r >> 40) * (1.0f / 16777216.0f); }

/* ------------------------------------------------------------------------ */
/* exp(x) for the acceptance test: Cody-Waite reduction x = k ln2 + r with   */
/* ln2 split in two parts, |r| <= ln2/2, then the Taylor series of e^r to    */
/* degree 20 (truncation error below 2^-70 relative), then scaling by 2^k.   */
/* ------------------------------------------------------------------------ */
double oracle_exp(double x) {
    if (x != x) return x;
    if (x > 709.0) return INFINITY;
    if (x < -708.0) return 0.0;
    const double ln2_hi = 0.693147180369123816490;     /* 32 significant bits of ln 2 */
    const double ln2_lo = 1.90821492927058770002e-10;  /* ln 2 - ln2_hi */
    const double inv_ln2 = 1.44269504088896338700;
    double kd = floor(x * inv_ln2 + 0.5);
    int k = (int)kd;
    double r = (x - kd * ln2_hi) - kd * ln2_lo;
    /* Horner from the highest term: sum_{j=0..20} r^j / j! */
    double s = 1.0;
    for (int j = 20; j >= 1; j--) s = 1.0 + s * (r / (double)j);
    /* 2^k for -1022 <= k <= 1023 built from its exponent field */
    union { uint64_t u; double f; } scale;
    scale.u = (uint64_t)(k + 1023) << 52;
    return s * scale.f;
}

/* ------------------------------------------------------------------------ */
/* Evaluation core with caller scratch, plus route travel (sum of legs).     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int cap_ops, cap_m;
    int32_t *ops, *off;      /* candidate build buffer */
    int32_t *ops2, *off2;
} scratch_t;

static int64_t Dd(const oracle_inst* I, int a, int b) { return I->d[(int64_t)a * (I->n + 1) + b]; }

static int64_t travel_of(const oracle_inst* I, const int32_t* ops, const int32_t* off) {
    int64_t t = 0;
    for (int v = 0; v < I->m; v++) {
        if (off[v + 1] == off[v]) continue;
        int loc = 0;
        for (int k = off[v]; k < off[v + 1]; k++) { t += Dd(I, loc, ops[k] >> 1); loc = ops[k] >> 1; }
        t += Dd(I, loc, 0);
    }
    return t;
}

/* Build S' = S + D_c at gap i of route a + P_c at gap j of route b. */
static void build_insert(const oracle_inst* I, const int32_t* ops, const int32_t* off, int c,
                         int a, int i, int b, int j, int32_t* nops, int32_t* noff) {
    int w = 0;
    noff[0] = 0;
    for (int v = 0; v < I->m; v++) {
        int L = off[v + 1] - off[v];
        for (int k = 0; k <= L; k++) {
            if (v == a && k == i) nops[w++] = 2 * c;
            if (v == b && k == j) nops[w++] = 2 * c + 1;
            if (k < L) nops[w++] = ops[off[v] + k];
        }
        noff[v + 1] = w;
    }
}

/* Capacity of one route (Eqs. 13-18 with the minimal or the full start load). */
static int route_cap_violated(const oracle_inst* I, const int32_t* ops, const int32_t* off, int v) {
    int64_t s = 0, smin = 0, smax = 0;
    for (int k = off[v]; k < off[v + 1]; k++) {
        s += (ops[k] & 1) ? 1 : -1;
        if (s < smin) smin = s;
        if (s > smax) smax = s;
    }
    if (I->flags & OR_LOAD_FULL) return smin < -(int64_t)I->Q || smax > 0;
    return -smin + smax > I->Q;
}

static int64_t pack_key_less(int64_t dz1, int64_t dt1, int64_t f1, int64_t dz2, int64_t dt2, int64_t f2) {
    if (dz1 != dz2) return dz1 < dz2;
    if (dt1 != dt2) return dt1 < dt2;
    return f1 < f2;
}

int oracle_insertion_matrix(const oracle_inst* I, const int32_t* ops, const int32_t* off,
                            int32_t c, int32_t* out, int32_t* travel_out, uint32_t* status_out) {
    const int m = I->m, N = off[m], G = N + m;
    int32_t z0;
    uint32_t st0;
    oracle_evaluate(I, ops, off, 1, &z0, &st0, NULL);
    if (st0 & (OR_CYCLE | OR_MALFORMED)) return -1;
    int64_t t0 = travel_of(I, ops, off);
    int32_t* nops = (int32_t*)malloc(sizeof(int32_t) * (N + 2));
    int32_t* noff = (int32_t*)malloc(sizeof(int32_t) * (m + 1));
    int rowbase = 0;
    for (int a = 0; a < m; a++) {
        int La = off[a + 1] - off[a];
        for (int i = 0; i <= La; i++) {
            int row = rowbase + i;
            int colbase = 0;
            for (int b = 0; b < m; b++) {
                int Lb = off[b + 1] - off[b];
                for (int j = 0; j <= Lb; j++) {
                    int col = colbase + j;
                    int64_t idx = (int64_t)row * G + col;
                    int32_t z;
                    uint32_t st;
                    if (a == b && j < i) {
                        /* pickup before its own drop on one route: a precedence cycle */
                        z = INT32_MAX;
                        st = OR_CYCLE;
                        if (travel_out) travel_out[idx] = 0;
                    } else {
                        build_insert(I, ops, off, c, a, i, b, j, nops, noff);
                        oracle_evaluate(I, nops, noff, 1, &z, &st, NULL);
                        /* vehicle capacity is judged on the two receiving routes only: a
                         * destroyed partial solution may violate it elsewhere */
                        st &= ~OR_VEH_CAP;
                        if (route_cap_violated(I, nops, noff, a) || route_cap_violated(I, nops, noff, b))
                            st |= OR_VEH_CAP;
                        if (travel_out) travel_out[idx] = (int32_t)(travel_of(I, nops, noff) - t0);
                    }
                    out[idx] = st ? INT32_MAX : (int32_t)(z - z0);
                    if (status_out) status_out[idx] = st;
                }
                colbase += Lb + 1;
            }
        }
        rowbase += La + 1;
    }
    free(nops);
    free(noff);
    return 0;
}

void oracle_q_range(int32_t n, int32_t* q_min, int32_t* q_max) {
    /* Section 4.2.2: q_max = max(4, floor(0.05 n)), q_min = max(4, floor(q_max/2)) */
    int32_t qm = (int32_t)((int64_t)n * 5 / 100);
    if (qm < 4) qm = 4;
    int32_t qn = qm / 2;
    if (qn < 4) qn = 4;
    *q_max = qm;
    *q_min = qn;
}

/* ------------------------------------------------------------------------ */
/* Initial solution: customers in exact angular order around the depot       */
/* (ties by customer id), split into m consecutive sectors by workload       */
/* w_c = 2 d(0,c) + p_c (midpoint rule), then each route serves its sector   */
/* in blocks of b customers as "D c1..cb, P c1..cb" with b = min(Q, R/m').   */
/* ------------------------------------------------------------------------ */
static const int32_t* g_coords;
static int angle_half(int64_t dx, int64_t dy) { return (dy < 0 || (dy == 0 && dx < 0)) ? 1 : 0; }
static int angle_cmp(const void* pa, const void* pb) {
    int a = *(const int*)pa, b = *(const int*)pb;
    int64_t ax = g_coords[2 * a] - g_coords[0], ay = g_coords[2 * a + 1] - g_coords[1];
    int64_t bx = g_coords[2 * b] - g_coords[0], by = g_coords[2 * b + 1] - g_coords[1];
    int ha = angle_half(ax, ay), hb = angle_half(bx, by);
    if (ha != hb) return ha - hb;
    int64_t cr = ax * by - ay * bx;
    if (cr > 0) return -1;
    if (cr < 0) return 1;
    return a - b;
}

int oracle_initial_solution(const oracle_inst* I, const int32_t* coords, int32_t* ops, int32_t* off) {
    const int n = I->n, m = I->m;
    if (I->R < 1 || I->Q < 1 || m < 1) return -1;
    int* order = (int*)malloc(sizeof(int) * (n + 1));
    for (int k = 0; k < n; k++) order[k] = k + 1;
    if (coords) {
        g_coords = coords;
        qsort(order, (size_t)n, sizeof(int), angle_cmp);
    }
    int mact = m < I->R ? m : I->R;
    int b = I->R / mact;
    if (b > I->Q) b = I->Q;
    if (b < 1) b = 1;
    int64_t W = 0;
    for (int k = 0; k < n; k++) W += 2 * Dd(I, 0, order[k]) + I->p[order[k] - 1];
    int* sector = (int*)malloc(sizeof(int) * (n + 1));
    int64_t cum = 0;
    for (int k = 0; k < n; k++) {
        int64_t w = 2 * Dd(I, 0, order[k]) + I->p[order[k] - 1];
        int64_t s = W > 0 ? ((2 * cum + w) * mact) / (2 * W) : ((int64_t)k * mact) / n;
        if (s > mact - 1) s = mact - 1;
        sector[k] = (int)s;
        cum += w;
    }
    int w = 0;
    off[0] = 0;
    for (int v = 0; v < m; v++) {
        int k = 0;
        while (k < n) {
            if (sector[k] != v) { k++; continue; }
            int blk[4096];
            int cnt = 0;
            while (k < n && cnt < b) {
                if (sector[k] == v) blk[cnt++] = order[k];
                k++;
            }
            for (int t = 0; t < cnt; t++) ops[w++] = 2 * blk[t];
            for (int t = 0; t < cnt; t++) ops[w++] = 2 * blk[t] + 1;
        }
        off[v + 1] = w;
    }
    free(order);
    free(sector);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* ALNS (Algorithm 1) with random removal and greedy / regret-2 repair.      */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t dz, dt, flat;
    int row, col, ok;
} best_t;

static void remove_customers(int m, const int32_t* ops, const int32_t* off, const char* rem,
                             int32_t* nops, int32_t* noff) {
    int w = 0;
    noff[0] = 0;
    for (int v = 0; v < m; v++) {
        for (int k = off[v]; k < off[v + 1]; k++)
            if (!rem[ops[k] >> 1]) nops[w++] = ops[k];
        noff[v + 1] = w;
    }
}

static void gap_of(const int32_t* off, int m, int g, int* route, int* pos) {
    for (int v = 0; v < m; v++) {
        int L = off[v + 1] - off[v];
        if (g <= L) { *route = v; *pos = g; return; }
        g -= L + 1;
    }
    *route = -1;
    *pos = -1;
}

/* Scan the matrix of customer c: overall best and per-drop-vehicle best. */
static void scan_matrix(const oracle_inst* I, const int32_t* ops, const int32_t* off, int c,
                        best_t* best, best_t* per_vehicle) {
    const int m = I->m, N = off[m], G = N + m;
    int32_t* M = (int32_t*)malloc(sizeof(int32_t) * (size_t)G * G);
    int32_t* T = (int32_t*)malloc(sizeof(int32_t) * (size_t)G * G);
    oracle_insertion_matrix(I, ops, off, c, M, T, NULL);
    best->ok = 0;
    for (int v = 0; v < m; v++) per_vehicle[v].ok = 0;
    for (int row = 0; row < G; row++) {
        int a, i;
        gap_of(off, m, row, &a, &i);
        for (int col = 0; col < G; col++) {
            int64_t idx = (int64_t)row * G + col;
            if (M[idx] == INT32_MAX) continue;
            int64_t dz = M[idx], dt = T[idx];
            if (!best->ok || pack_key_less(dz, dt, idx, best->dz, best->dt, best->flat))
                *best = (best_t){dz, dt, idx, row, col, 1};
            best_t* pv = &per_vehicle[a];
            if (!pv->ok || pack_key_less(dz, dt, idx, pv->dz, pv->dt, pv->flat))
                *pv = (best_t){dz, dt, idx, row, col, 1};
        }
    }
    free(M);
    free(T);
}

static void apply_insert(const oracle_inst* I, int32_t* ops, int32_t* off, int c, int row, int col,
                         int32_t* tmp_ops, int32_t* tmp_off) {
    int a, i, b, j;
    gap_of(off, I->m, row, &a, &i);
    gap_of(off, I->m, col, &b, &j);
    build_insert(I, ops, off, c, a, i, b, j, tmp_ops, tmp_off);
    memcpy(ops, tmp_ops, sizeof(int32_t) * tmp_off[I->m]);
    memcpy(off, tmp_off, sizeof(int32_t) * (I->m + 1));
}

#define REGRET_INF ((int64_t)1 << 40)

/* Greedy (repair 0) or regret-k (repair 1, 2, 3: k = 2, 3, m) reinsertion of
 * the customers listed in ascending id order in list[]: one insertion per
 * step, at most max_steps steps (negative: until none is left). */
static int repair_steps(const oracle_inst* I, int op, int32_t* ops, int32_t* off, int* list, int cnt,
                        int max_steps, int32_t* tmp_ops, int32_t* tmp_off) {
    const int m = I->m;
    best_t* pv = (best_t*)malloc(sizeof(best_t) * m);
    best_t* bests = (best_t*)malloc(sizeof(best_t) * (cnt + 1));
    int64_t* regret = (int64_t*)malloc(sizeof(int64_t) * (cnt + 1));
    for (int step = 0; cnt > 0 && step != max_steps; step++) {
        for (int t = 0; t < cnt; t++) {
            scan_matrix(I, ops, off, list[t], &bests[t], pv);
            if (!bests[t].ok) { free(pv); free(bests); free(regret); return -1; }
            /* regret-k (Section 4.2.3): the options are the best insertion per
             * dropoff vehicle (REGRET_INF where a vehicle has none); regret =
             * sum over the k best of (c_i - c_1), options past the m there are
             * counting as REGRET_INF.  k = 2, 3 or m for operators 1, 2, 3. */
            int64_t cs[64];
            for (int v = 0; v < m; v++) cs[v] = pv[v].ok ? pv[v].dz : REGRET_INF;
            for (int i = 1; i < m; i++)                                     /* insertion sort */
                for (int j = i; j > 0 && cs[j] < cs[j - 1]; j--) { int64_t x = cs[j]; cs[j] = cs[j - 1]; cs[j - 1] = x; }
            const int k = op == 1 ? 2 : (op == 2 ? 3 : m);
            int64_t r = 0;
            for (int i = 0; i < k; i++) r += (i < m ? cs[i] : REGRET_INF) - cs[0];
            regret[t] = r;
        }
        int pick = 0;
        for (int t = 1; t < cnt; t++) {
            if (op == 0) {
                /* greedy: smallest key; equal keys -> smaller customer id (list is ascending) */
                if (pack_key_less(bests[t].dz, bests[t].dt, bests[t].flat, bests[pick].dz, bests[pick].dt,
                                  bests[pick].flat))
                    pick = t;
            } else {
                /* regret-k: largest regret; ties -> smaller customer id */
                if (regret[t] > regret[pick]) pick = t;
            }
        }
        apply_insert(I, ops, off, list[pick], bests[pick].row, bests[pick].col, tmp_ops, tmp_off);
        for (int t = pick; t + 1 < cnt; t++) list[t] = list[t + 1];
        cnt--;
    }
    free(pv);
    free(bests);
    free(regret);
    return 0;
}

static int repair(const oracle_inst* I, int op, int32_t* ops, int32_t* off, int* list, int cnt,
                  int32_t* tmp_ops, int32_t* tmp_off) {
    return repair_steps(I, op, ops, off, list, cnt, -1, tmp_ops, tmp_off);
}

int oracle_repair(const oracle_inst* I, int32_t op, const int32_t* ops, const int32_t* off, const int32_t* removed,
                  int32_t count, int32_t max_steps, int32_t* out_ops, int32_t* out_off) {
    const int m = I->m, N = off[m];
    if (op < 0 || op > 3 || count < 0 || N + 2 * count > 2 * I->n) return -1;
    int* list = malloc(sizeof(int) * (size_t)(count + 1));
    for (int t = 0; t < count; t++) {
        if (removed[t] < 1 || removed[t] > I->n || (t > 0 && removed[t] <= removed[t - 1])) { free(list); return -1; }
        list[t] = removed[t];
    }
    int32_t* tmp = malloc(sizeof(int32_t) * (size_t)(2 * I->n + 2));
    int32_t* tmpo = malloc(sizeof(int32_t) * (size_t)(m + 1));
    memcpy(out_ops, ops, sizeof(int32_t) * (size_t)N);
    memcpy(out_off, off, sizeof(int32_t) * (size_t)(m + 1));
    int rc = repair_steps(I, op, out_ops, out_off, list, count, max_steps, tmp, tmpo);
    free(list);
    free(tmp);
    free(tmpo);
    return rc;
}

static int roulette(const double* w, const int* enabled, int k, double u) {
    double sum = 0.0;
    for (int i = 0; i < k; i++)
        if (enabled[i]) sum += w[i];
    double target = u * sum, acc = 0.0;
    int last = -1;
    for (int i = 0; i < k; i++) {
        if (!enabled[i]) continue;
        acc += w[i];
        last = i;
        if (target < acc) return i;
    }
    return last;
}

/* ------------------------------------------------------------------------ */
/* Destroy operators (Section 4.2.2).  Each marks the customers to remove in   */
/* rem[] and returns how many.  Draws: operator-specific picks at counter      */
/* base + 4, sequential draws k at base + 16 + k.                              */
/* ------------------------------------------------------------------------ */
enum { D_RANDOM = 0, D_WORST = 1, D_SHAW = 2, D_CLUSTER = 3, D_ROUTE = 4, D_CRITICAL = 5, ND_OPS = 6 };

typedef struct {
    int64_t key;
    int c;
} rank_t;
static int rank_cmp(const void* pa, const void* pb) {
    const rank_t *a = pa, *b = pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return a->c - b->c;                             /* ties: the smaller customer id first */
}

/* facts of the current solution: departure per op code (drop: arrival), the
 * vehicles of each customer's dropoff and pickup, and each route's return time */
static void solution_facts(const oracle_inst* I, const int32_t* S, const int32_t* So, int64_t* times,
                           int* vd, int* vp, int64_t* ret) {
    int32_t z;
    uint32_t st;
    oracle_evaluate(I, S, So, 0, &z, &st, times);
    for (int v = 0; v < I->m; v++) {
        ret[v] = 0;
        for (int k = So[v]; k < So[v + 1]; k++) {
            int o = S[k];
            if (o & 1) vp[o >> 1] = v; else vd[o >> 1] = v;
        }
        if (So[v + 1] > So[v]) {
            int o = S[So[v + 1] - 1];
            ret[v] = times[o] + Dd(I, o >> 1, 0);
        }
    }
}

int oracle_destroy(const oracle_inst* I, int32_t di, const int32_t* S, const int32_t* So, int32_t q,
                   int32_t qmin, uint64_t key, uint64_t base, char* rem) {
    const int n = I->n, m = I->m, two_n = 2 * n;
    memset(rem, 0, (size_t)n + 1);
    int cnt = 0;
    if (di == D_RANDOM) {
        /* partial Fisher-Yates over customers 1..n */
        int* perm = malloc(sizeof(int) * (n + 1));
        for (int k = 0; k < n; k++) perm[k] = k + 1;
        for (int k = 0; k < q; k++) {
            int jj = k + rng_below(oracle_rng(key, base + 16 + (uint64_t)k), n - k);
            int t = perm[k]; perm[k] = perm[jj]; perm[jj] = t;
            rem[perm[k]] = 1;
        }
        free(perm);
        return q;
    }
    int64_t* times = malloc(sizeof(int64_t) * (two_n + 2));
    int* vd = calloc((size_t)n + 1, sizeof(int));
    int* vp = calloc((size_t)n + 1, sizeof(int));
    int64_t* ret = calloc((size_t)m, sizeof(int64_t));
    rank_t* rk = malloc(sizeof(rank_t) * (n + 1));
    solution_facts(I, S, So, times, vd, vp, ret);
    if (di == D_WORST) {
        /* removal gain z(S) - z(S - c); customers ranked by gain, largest
         * first; q roulette draws over the remaining ranked list with weight
         * r^-6 for the r-th remaining customer (power p = 6) */
        int32_t z, zc;
        uint32_t st;
        oracle_evaluate(I, S, So, 0, &z, &st, NULL);
        int32_t* T = malloc(sizeof(int32_t) * (two_n + 2));
        int32_t* To = malloc(sizeof(int32_t) * (m + 1));
        char* one = calloc((size_t)n + 1, 1);
        for (int c = 1; c <= n; c++) {
            one[c] = 1;
            remove_customers(m, S, So, one, T, To);
            one[c] = 0;
            oracle_evaluate(I, T, To, 1, &zc, &st, NULL);
            rk[c - 1].key = -((int64_t)z - (int64_t)zc);
            rk[c - 1].c = c;
        }
        free(T); free(To); free(one);
        qsort(rk, (size_t)n, sizeof(rank_t), rank_cmp);
        double* P = malloc(sizeof(double) * (n + 1));
        double acc = 0.0;
        for (int r = 1; r <= n; r++) {
            double x = (double)r, x2 = x * x;
            acc += 1.0 / (x2 * x2 * x2);
            P[r] = acc;
        }
        for (int k = 0; k < q; k++) {
            const int R = n - k;
            const double target = rng_unit(oracle_rng(key, base + 16 + (uint64_t)k)) * P[R];
            int r = 1;
            while (r < R && !(P[r] > target)) r++;
            /* the r-th customer of the ranked list not removed yet */
            int seen = 0;
            for (int i = 0; i < n; i++) {
                if (rem[rk[i].c]) continue;
                if (++seen == r) { rem[rk[i].c] = 1; break; }
            }
        }
        free(P);
        cnt = q;
    } else if (di == D_SHAW || di == D_CLUSTER) {
        /* a random seed customer and the q - 1 customers closest to it: by
         * 2R = 18 d + 6 |T_drop diff| + 5 [dropoff vehicles differ] + 5 [pickup
         * vehicles differ] (Shaw, phi 9, chi 3, omega 5), or by travel time
         * alone (cluster); ties to the smaller customer id */
        const int sd = 1 + rng_below(oracle_rng(key, base + 4), n);
        int w = 0;
        for (int c = 1; c <= n; c++) {
            if (c == sd) continue;
            int64_t k2 = Dd(I, sd, c);
            if (di == D_SHAW) {
                int64_t dt = times[2 * sd] - times[2 * c];
                if (dt < 0) dt = -dt;
                k2 = 18 * k2 + 6 * dt + 5 * (vd[sd] != vd[c]) + 5 * (vp[sd] != vp[c]);
            }
            rk[w].key = k2;
            rk[w].c = c;
            w++;
        }
        qsort(rk, (size_t)w, sizeof(rank_t), rank_cmp);
        rem[sd] = 1;
        for (int k = 0; k + 1 < q && k < w; k++) rem[rk[k].c] = 1;
        cnt = q < n ? q : n;
    } else if (di == D_ROUTE || di == D_CRITICAL) {
        int vsel = 0;
        if (di == D_ROUTE) {
            /* the k-th non-empty route */
            int K = 0;
            for (int v = 0; v < m; v++) K += So[v + 1] > So[v];
            int kk = rng_below(oracle_rng(key, base + 4), K);
            for (int v = 0; v < m; v++)
                if (So[v + 1] > So[v] && kk-- == 0) { vsel = v; break; }
            for (int k = So[vsel]; k < So[vsel + 1]; k++)
                if (!rem[S[k] >> 1]) { rem[S[k] >> 1] = 1; cnt++; }
        } else {
            /* the bottleneck route (latest return, the lower index on ties):
             * q of its customers, or all if fewer, by partial Fisher-Yates in
             * customer order */
            for (int v = 1; v < m; v++)
                if (ret[v] > ret[vsel]) vsel = v;
            int* L = malloc(sizeof(int) * (n + 1));
            int nl = 0;
            for (int c = 1; c <= n; c++)
                if (vd[c] == vsel || vp[c] == vsel) L[nl++] = c;
            int take = q < nl ? q : nl;
            for (int k = 0; k < take; k++) {
                int jj = k + rng_below(oracle_rng(key, base + 16 + (uint64_t)k), nl - k);
                int t = L[k]; L[k] = L[jj]; L[jj] = t;
                rem[L[k]] = 1;
            }
            cnt = take;
            free(L);
        }
        if (cnt < qmin) {
            /* top up from the other routes: route removal by the least travel
             * time from a removed customer, critical path by the latest pickup
             * completion; ties to the smaller customer id */
            int w = 0;
            for (int c = 1; c <= n; c++) {
                if (rem[c]) continue;
                int64_t k2;
                if (di == D_ROUTE) {
                    k2 = INT64_MAX;
                    for (int r = 1; r <= n; r++)
                        if (rem[r] && Dd(I, r, c) < k2) k2 = Dd(I, r, c);
                } else {
                    k2 = -times[2 * c + 1];
                }
                rk[w].key = k2;
                rk[w].c = c;
                w++;
            }
            qsort(rk, (size_t)w, sizeof(rank_t), rank_cmp);
            for (int k = 0; k < w && cnt < qmin; k++) { rem[rk[k].c] = 1; cnt++; }
        }
    }
    free(times); free(vd); free(vp); free(ret); free(rk);
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* Periodic local search (Section 4.2.6) on the current solution.            */
/*   LS_PICKUP:   pickup repositioning.  Candidates: customers whose pickup   */
/*                sits on a vehicle returning at 95% of the makespan or later */
/*                (20 ret >= 19 z).  Move: the pickup to any position of any  */
/*                vehicle, the dropoff left where it is.                      */
/*   LS_RELOCATE: cross-agent relocation.  Candidates: customers with an op   */
/*                on the bottleneck vehicle (latest return, lower index on   */
/*                ties).  Move: dropoff and pickup together onto one other    */
/*                vehicle, at any positions in that order.                    */
/* A pass scores every move of every candidate by the resulting solution:    */
/* (makespan, total travel, customer, flat gap index row*G + col, gaps of    */
/* the solution without the customer), feasible only with no status bit.    */
/* It applies the least if its makespan is below the current one; up to      */
/* three passes, candidates re-derived each time.  Returns the moves made.   */
/* ------------------------------------------------------------------------ */
enum { LS_PICKUP = 1, LS_RELOCATE = 2 };

static int local_search(const oracle_inst* I, int mode, int32_t* S, int32_t* So, int32_t* z, int passes) {
    const int n = I->n, m = I->m, two_n = 2 * n;
    int64_t* times = malloc(sizeof(int64_t) * (two_n + 2));
    int* vd = calloc((size_t)n + 1, sizeof(int));
    int* vp = calloc((size_t)n + 1, sizeof(int));
    int* pd = calloc((size_t)n + 1, sizeof(int));
    int64_t* ret = calloc((size_t)m, sizeof(int64_t));
    int32_t *W = malloc(sizeof(int32_t) * (two_n + 2)), *Wo = malloc(sizeof(int32_t) * (m + 1));
    int32_t *X = malloc(sizeof(int32_t) * (two_n + 2)), *Xo = malloc(sizeof(int32_t) * (m + 1));
    char* rem = calloc((size_t)n + 1, 1);
    int moves = 0;
    for (int pass = 0; pass < passes; pass++) {
        solution_facts(I, S, So, times, vd, vp, ret);
        for (int v = 0; v < m; v++)
            for (int k = So[v]; k < So[v + 1]; k++)
                if (!(S[k] & 1)) pd[S[k] >> 1] = k - So[v];
        const int64_t zc = *z;
        int bott = 0;
        for (int v = 1; v < m; v++)
            if (ret[v] > ret[bott]) bott = v;
        int have = 0, bc = 0, ba = 0, bi = 0, bb = 0, bj = 0;
        int64_t bz = 0, bt = 0, bf = 0;
        const int G = (two_n - 2) + m;
        for (int c = 1; c <= n; c++) {
            if (mode == LS_PICKUP ? !(20 * ret[vp[c]] >= 19 * zc) : (vd[c] != bott && vp[c] != bott)) continue;
            rem[c] = 1;
            remove_customers(m, S, So, rem, W, Wo);
            rem[c] = 0;
            for (int a = 0; a < m; a++) {
                if (mode == LS_PICKUP && a != vd[c]) continue;
                if (mode == LS_RELOCATE && a == bott) continue;
                const int La = Wo[a + 1] - Wo[a];
                for (int i = 0; i <= La; i++) {
                    if (mode == LS_PICKUP && i != pd[c]) continue;
                    for (int b = 0; b < m; b++) {
                        if (mode == LS_RELOCATE && b != a) continue;
                        const int Lb = Wo[b + 1] - Wo[b];
                        for (int j = (b == a ? i : 0); j <= Lb; j++) {
                            build_insert(I, W, Wo, c, a, i, b, j, X, Xo);
                            int32_t zn;
                            uint32_t st;
                            oracle_evaluate(I, X, Xo, 0, &zn, &st, NULL);
                            if (st) continue;
                            const int64_t tn = travel_of(I, X, Xo);
                            const int64_t flat = (int64_t)(Wo[a] + a + i) * G + (Wo[b] + b + j);
                            int better = !have;
                            if (!better) {
                                if (zn != bz) better = zn < bz;
                                else if (tn != bt) better = tn < bt;
                                else if (c != bc) better = c < bc;
                                else better = flat < bf;
                            }
                            if (better) {
                                have = 1;
                                bz = zn; bt = tn; bc = c; bf = flat;
                                ba = a; bi = i; bb = b; bj = j;
                            }
                        }
                    }
                }
            }
        }
        if (!have || bz >= zc) break;
        rem[bc] = 1;
        remove_customers(m, S, So, rem, W, Wo);
        rem[bc] = 0;
        build_insert(I, W, Wo, bc, ba, bi, bb, bj, X, Xo);
        memcpy(S, X, sizeof(int32_t) * two_n);
        memcpy(So, Xo, sizeof(int32_t) * (m + 1));
        *z = (int32_t)bz;
        moves++;
    }
    free(times); free(vd); free(vp); free(pd); free(ret); free(W); free(Wo); free(X); free(Xo); free(rem);
    return moves;
}

int oracle_local_search(const oracle_inst* I, int32_t mode, int32_t passes, int32_t* ops, int32_t* off,
                        int32_t* z) {
    int32_t z0;
    uint32_t st;
    oracle_evaluate(I, ops, off, 0, &z0, &st, NULL);
    if (st || (mode != LS_PICKUP && mode != LS_RELOCATE)) return -1;
    *z = z0;
    return local_search(I, mode, ops, off, z, passes);
}

/* One ALNS instance (Algorithm 1) as resumable state: its solutions, the
 * temperature, the operator weights and scores, and its draw stream. */
typedef struct {
    const oracle_inst* I;
    const oracle_alns_params* P;
    int32_t *S, *So, *Sb, *Sbo, *W, *Wo, *tmp, *tmpo;
    int* list;
    char* rem;
    int32_t z, zb, qmin, qmax;
    uint64_t key;
    double wd[ND_OPS], wr[4], T, T_init;
    int sd[ND_OPS], sr[4], ad[ND_OPS], ar[4], en_d[ND_OPS], en_r[4];
    int stagnation;
    oracle_alns_stats* stats;
    int32_t* z_trace;
} alns_t;

static int alns_init(alns_t* A, const oracle_inst* I, const int32_t* init_ops, const int32_t* init_off,
                     const oracle_alns_params* P, uint64_t key, oracle_alns_stats* stats, int32_t* z_trace) {
    const int n = I->n, m = I->m, two_n = 2 * n;
    memset(A, 0, sizeof(*A));
    A->I = I;
    A->P = P;
    A->S = malloc(sizeof(int32_t) * two_n); A->So = malloc(sizeof(int32_t) * (m + 1));
    A->Sb = malloc(sizeof(int32_t) * two_n); A->Sbo = malloc(sizeof(int32_t) * (m + 1));
    A->W = malloc(sizeof(int32_t) * (two_n + 2)); A->Wo = malloc(sizeof(int32_t) * (m + 1));
    A->tmp = malloc(sizeof(int32_t) * (two_n + 2)); A->tmpo = malloc(sizeof(int32_t) * (m + 1));
    A->list = malloc(sizeof(int) * (n + 1));
    A->rem = calloc((size_t)n + 1, 1);
    memcpy(A->S, init_ops, sizeof(int32_t) * two_n);
    memcpy(A->So, init_off, sizeof(int32_t) * (m + 1));
    uint32_t st;
    oracle_evaluate(I, A->S, A->So, 0, &A->z, &st, NULL);
    if (st) return -2;                             /* the search starts from a feasible solution */
    memcpy(A->Sb, A->S, sizeof(int32_t) * two_n);
    memcpy(A->Sbo, A->So, sizeof(int32_t) * (m + 1));
    A->zb = A->z;
    A->key = key;
    A->qmin = P->q_min;
    A->qmax = P->q_max;
    if (A->qmin <= 0 || A->qmax <= 0) oracle_q_range(n, &A->qmin, &A->qmax);
    if (A->qmax > n) A->qmax = n;
    if (A->qmin > A->qmax) A->qmin = A->qmax;
    /* operators: destroy 0 random, 1 worst, 2 Shaw, 3 cluster, 4 route, 5
     * critical path (destroy_mask bits); repair 0 greedy, 1 regret-2, 2
     * regret-3, 3 regret-m (repair_mask bits) */
    for (int i = 0; i < ND_OPS; i++) { A->wd[i] = 1.0; A->en_d[i] = (P->destroy_mask >> i) & 1; }
    for (int i = 0; i < 4; i++) { A->wr[i] = 1.0; A->en_r[i] = (P->repair_mask >> i) & 1; }
    A->T = P->T0 * (double)A->z;                   /* initial temperature */
    A->T_init = A->T;
    A->stats = stats;
    A->z_trace = z_trace;
    memset(stats, 0, sizeof(*stats));
    stats->z_init = A->z;
    return 0;
}

/* Algorithm 1's bookkeeping of iteration it once the repair is done: destroy
 * operator di and repair operator rj gave a candidate of makespan zn and
 * status st, and u is the iteration's SA draw.  A candidate with a status bit
 * is rejected.  One below the current makespan is accepted and scores sigma2,
 * or sigma1 if it is also below the best.  Any other is accepted when
 * u < exp(-(zn - z)/T) and scores sigma3 (an equal makespan gives exp(0) = 1).
 * Then cooling T <- alpha T, the stagnation count, the reheat (stagnation and
 * T below 1% of its start: T <- reheat T0 z_best) and, every tau iterations,
 * w <- max(w_min, (1 - r) w + r s/a) per operator (s/a = 0 without attempts).
 * Returns 0 (rejected), 1 (current) or 2 (current and new best). */
static int alns_accept_adapt(alns_t* A, int it, int di, int rj, int32_t zn, uint32_t st, double u) {
    const oracle_alns_params* P = A->P;
    oracle_alns_stats* stats = A->stats;
    const int ND = ND_OPS, NR = 4;
    int took = 0;
    A->ad[di]++;
    A->ar[rj]++;                                                                 /* attempt counts */
    if (st) {
        /* repair found no feasible slot, or a route the destroy left over
         * capacity was never repaired: the candidate is rejected */
        stats->rejected_infeasible++;
    } else if (zn < A->z) {                                                      /* improving: accept, scores */
        A->z = zn;
        A->sd[di] += P->sigma2;
        A->sr[rj] += P->sigma2;
        stats->improved++;
        stats->accepted++;
        took = 1;
        if (zn < A->zb) {
            A->zb = zn;
            A->sd[di] += P->sigma1 - P->sigma2;
            A->sr[rj] += P->sigma1 - P->sigma2;
            A->stagnation = 0;
            stats->new_best++;
            took = 2;
        }
    } else {
        double x = -(double)((int64_t)zn - (int64_t)A->z) / A->T;
        if (u < oracle_exp(x)) {                                                 /* SA acceptance */
            A->z = zn;
            A->sd[di] += P->sigma3;
            A->sr[rj] += P->sigma3;
            stats->accepted++;
            took = 1;
        }
    }
    A->T = P->alpha * A->T;                                                      /* cooling */
    A->stagnation++;                                                             /* stagnation count */
    if (A->stagnation >= P->stagnation && A->T < 0.01 * A->T_init) {             /* reheat, with the text's temperature gate */
        A->T = (P->reheat * P->T0) * (double)A->zb;
        A->stagnation = 0;
        stats->reheats++;
    }
    if (it % P->tau == 0) {                                                      /* weight update every tau */
        for (int i = 0; i < ND; i++) {
            double ratio = A->ad[i] ? (double)A->sd[i] / (double)A->ad[i] : 0.0;
            double w = (1.0 - P->r) * A->wd[i] + P->r * ratio;
            A->wd[i] = w < P->w_min ? P->w_min : w;
            A->sd[i] = 0;
            A->ad[i] = 0;
        }
        for (int i = 0; i < NR; i++) {
            double ratio = A->ar[i] ? (double)A->sr[i] / (double)A->ar[i] : 0.0;
            double w = (1.0 - P->r) * A->wr[i] + P->r * ratio;
            A->wr[i] = w < P->w_min ? P->w_min : w;
            A->sr[i] = 0;
            A->ar[i] = 0;
        }
    }
    return took;
}

/* Iteration it of Algorithm 1, then the periodic local search. */
static void alns_iteration(alns_t* A, int it) {
    const oracle_inst* I = A->I;
    const oracle_alns_params* P = A->P;
    const int n = I->n, m = I->m, two_n = 2 * n, ND = ND_OPS, NR = 4;
    oracle_alns_stats* stats = A->stats;
    const uint64_t base = (uint64_t)it << 16, key = A->key;
    int di = roulette(A->wd, A->en_d, ND, rng_unit(oracle_rng(key, base + 0)));   /* destroy operator by roulette */
    int rj = roulette(A->wr, A->en_r, NR, rng_unit(oracle_rng(key, base + 1)));   /* repair operator by roulette */
    int q = A->qmin + rng_below(oracle_rng(key, base + 2), A->qmax - A->qmin + 1);
    oracle_destroy(I, di, A->S, A->So, q, A->qmin, key, base, A->rem);           /* destroy */
    remove_customers(m, A->S, A->So, A->rem, A->W, A->Wo);
    int cnt = 0;
    for (int c = 1; c <= n; c++)
        if (A->rem[c]) A->list[cnt++] = c;
    int32_t zn = INT32_MAX;
    uint32_t st = OR_MALFORMED;
    if (repair(I, rj, A->W, A->Wo, A->list, cnt, A->tmp, A->tmpo) == 0)          /* repair */
        oracle_evaluate(I, A->W, A->Wo, 0, &zn, &st, NULL);                      /* makespan of the candidate */
    const int took = alns_accept_adapt(A, it, di, rj, zn, st, rng_unit(oracle_rng(key, base + 3)));
    if (took >= 1) {                                                             /* the candidate is current */
        memcpy(A->S, A->W, sizeof(int32_t) * two_n);
        memcpy(A->So, A->Wo, sizeof(int32_t) * (m + 1));
    }
    if (took == 2) {                                                             /* and the new best */
        memcpy(A->Sb, A->W, sizeof(int32_t) * two_n);
        memcpy(A->Sbo, A->Wo, sizeof(int32_t) * (m + 1));
    }
    /* periodic local search on the current solution (Section 4.2.6):
     * pickup repositioning first when both fall due */
    if (P->ls_pickup_every > 0 && it % P->ls_pickup_every == 0)
        stats->ls_moves += local_search(I, LS_PICKUP, A->S, A->So, &A->z, 3);
    if (P->ls_relocate_every > 0 && it % P->ls_relocate_every == 0)
        stats->ls_moves += local_search(I, LS_RELOCATE, A->S, A->So, &A->z, 3);
    if (A->z < A->zb) {
        memcpy(A->Sb, A->S, sizeof(int32_t) * two_n);
        memcpy(A->Sbo, A->So, sizeof(int32_t) * (m + 1));
        A->zb = A->z;
        A->stagnation = 0;
        stats->ls_new_best++;
    }
    if (A->z_trace) A->z_trace[it - 1] = A->z;
    stats->iterations = it;
}

static void alns_finish(alns_t* A, int32_t* cur_ops_out, int32_t* cur_off_out) {
    const int two_n = 2 * A->I->n, m = A->I->m;
    if (cur_ops_out) memcpy(cur_ops_out, A->S, sizeof(int32_t) * two_n);
    if (cur_off_out) memcpy(cur_off_out, A->So, sizeof(int32_t) * (m + 1));
    A->stats->z_best = A->zb;
    A->stats->z_current = A->z;
    A->stats->T_final = A->T;
    for (int i = 0; i < ND_OPS; i++) A->stats->w_destroy[i] = A->wd[i];
    for (int i = 0; i < 4; i++) A->stats->w_repair[i] = A->wr[i];
}

static void alns_free(alns_t* A) {
    free(A->S); free(A->So); free(A->Sb); free(A->Sbo); free(A->W); free(A->Wo); free(A->tmp); free(A->tmpo);
    free(A->list); free(A->rem);
}

int oracle_alns_run(const oracle_inst* I, const int32_t* init_ops, const int32_t* init_off,
                    const oracle_alns_params* P, uint64_t seed, int32_t* best_ops, int32_t* best_off,
                    int32_t* cur_ops_out, int32_t* cur_off_out, oracle_alns_stats* stats,
                    int32_t* z_trace) {
    alns_t A;
    if (alns_init(&A, I, init_ops, init_off, P, stream_key(seed, STREAM_ALNS), stats, z_trace)) {
        alns_free(&A);
        return -2;
    }
    for (int it = 1; it <= P->iterations; it++) alns_iteration(&A, it);
    alns_finish(&A, cur_ops_out, cur_off_out);
    memcpy(best_ops, A.Sb, sizeof(int32_t) * 2 * I->n);
    memcpy(best_off, A.Sbo, sizeof(int32_t) * (I->m + 1));
    alns_free(&A);
    return 0;
}

int oracle_alns_adapt_script(const oracle_alns_params* P, int32_t z0, int32_t iters, const int32_t* di,
                             const int32_t* rj, const int32_t* zn, const uint32_t* st, const double* u,
                             oracle_alns_stats* stats, int32_t* z_trace) {
    alns_t A;
    memset(&A, 0, sizeof(A));
    memset(stats, 0, sizeof(*stats));
    A.P = P;
    A.stats = stats;
    A.z = A.zb = z0;
    for (int i = 0; i < ND_OPS; i++) A.wd[i] = 1.0;
    for (int i = 0; i < 4; i++) A.wr[i] = 1.0;
    A.T = P->T0 * (double)z0;                      /* initial temperature, as alns_init */
    A.T_init = A.T;
    stats->z_init = z0;
    for (int it = 1; it <= iters; it++) {
        if (di[it - 1] < 0 || di[it - 1] >= ND_OPS || rj[it - 1] < 0 || rj[it - 1] >= 4) return -1;
        alns_accept_adapt(&A, it, di[it - 1], rj[it - 1], zn[it - 1], st[it - 1], u[it - 1]);
        if (z_trace) z_trace[it - 1] = A.z;
        stats->iterations = it;
    }
    stats->z_best = A.zb;
    stats->z_current = A.z;
    stats->T_final = A.T;
    for (int i = 0; i < ND_OPS; i++) stats->w_destroy[i] = A.wd[i];
    for (int i = 0; i < 4; i++) stats->w_repair[i] = A.wr[i];
    return 0;
}

/* The draw stream of replica r: the ALNS stream itself for r = 0, else a
 * draw of it far past any iteration's counters. */
static uint64_t replica_key(uint64_t key0, int r) {
    return r == 0 ? key0 : oracle_rng(key0, (0xFFFFFFFFull << 32) + (uint64_t)r);
}

int oracle_alns_run_replicas(const oracle_inst* I, const int32_t* init_ops, const int32_t* init_off,
                             const oracle_alns_params* P, uint64_t seed, int32_t replicas, int32_t sync_every,
                             int32_t* best_ops, int32_t* best_off, int32_t* best_replica,
                             oracle_alns_stats* stats, int32_t* z_traces, int32_t* imports) {
    const int n = I->n, m = I->m;
    alns_t* A = calloc((size_t)replicas, sizeof(alns_t));
    const uint64_t key0 = stream_key(seed, STREAM_ALNS);
    int rc = 0;
    for (int r = 0; r < replicas && !rc; r++)
        rc = alns_init(&A[r], I, init_ops, init_off, P, replica_key(key0, r), &stats[r],
                       z_traces ? z_traces + (size_t)r * P->iterations : NULL);
    *imports = 0;
    for (int it = 1; it <= P->iterations && !rc; it++) {
        for (int r = 0; r < replicas; r++) alns_iteration(&A[r], it);
        if (replicas > 1 && sync_every > 0 && it % sync_every == 0) {
            /* every replica takes the best of all when its own is worse (the
             * lowest index among equal bests) */
            int g = 0;
            for (int r = 1; r < replicas; r++)
                if (A[r].zb < A[g].zb) g = r;
            for (int r = 0; r < replicas; r++) {
                if (A[r].zb <= A[g].zb) continue;
                memcpy(A[r].S, A[g].Sb, sizeof(int32_t) * 2 * n);
                memcpy(A[r].So, A[g].Sbo, sizeof(int32_t) * (m + 1));
                memcpy(A[r].Sb, A[g].Sb, sizeof(int32_t) * 2 * n);
                memcpy(A[r].Sbo, A[g].Sbo, sizeof(int32_t) * (m + 1));
                A[r].z = A[r].zb = A[g].zb;
                A[r].stagnation = 0;
                (*imports)++;
            }
        }
    }
    if (!rc) {
        int g = 0;
        for (int r = 0; r < replicas; r++) {
            alns_finish(&A[r], NULL, NULL);
            if (A[r].zb < A[g].zb) g = r;
        }
        memcpy(best_ops, A[g].Sb, sizeof(int32_t) * 2 * n);
        memcpy(best_off, A[g].Sbo, sizeof(int32_t) * (m + 1));
        *best_replica = g;
    }
    for (int r = 0; r < replicas; r++) alns_free(&A[r]);
    free(A);
    return rc ? -2 : 0;
}

/* The paper's three-phase constructor (Section 4.2.5), then its refinement.
 *   1. sweep: customers by exact angle around the depot (coordinates; without
 *      coordinates, by id), cut into m' = min(m, R) sectors of equal count
 *      (customer k of the order goes to sector floor(k m' / n));
 *   2. load balancing on w_c = 2 d(0,c) + p_c: while 10 m' (W_max - W_min) >=
 *      sum W (imbalance of 10% of the mean or more), the heaviest sector
 *      (lowest index on ties) hands its boundary customer to its lighter
 *      neighbour (lower index on ties), unless that would leave the
 *      neighbour at least as heavy as the heaviest was; at most 4n moves;
 *   3. nearest-neighbour routes: vehicle v serves its sector alone, starting
 *      at the depot at time 0 with b = min(Q, floor(R / m')) resources; at
 *      each step it takes the feasible op that completes first (a drop if a
 *      resource is left: arrival; a pickup of a dropped customer: max(arrival,
 *      T_drop + p)), ties by travel, then drop before pickup, then id.
 *   Refinement: rounds of pickup repositioning then cross-agent relocation
 *   (the periodic local search, three passes each) until a round moves
 *   nothing, at most refine_rounds rounds.
 * Feasible by construction: one vehicle per customer, at most b outstanding. */
int oracle_initial_solution_paper(const oracle_inst* I, const int32_t* coords, int32_t refine_rounds,
                                  int32_t* ops, int32_t* off) {
    const int n = I->n, m = I->m;
    if (I->R < 1 || I->Q < 1 || m < 1) return -1;
    int* order = malloc(sizeof(int) * (n + 1));
    for (int k = 0; k < n; k++) order[k] = k + 1;
    if (coords) {
        g_coords = coords;
        qsort(order, (size_t)n, sizeof(int), angle_cmp);
    }
    const int mp = m < I->R ? m : I->R;
    int b = I->R / mp;
    if (b > I->Q) b = I->Q;
    int* start = calloc((size_t)mp + 1, sizeof(int));
    int64_t* Wl = calloc((size_t)mp, sizeof(int64_t));
    for (int k = 0; k < n; k++) {
        const int sct = (int)(((int64_t)k * mp) / n);
        Wl[sct] += 2 * Dd(I, 0, order[k]) + I->p[order[k] - 1];
    }
    for (int sct = 0; sct <= mp; sct++) start[sct] = (int)(((int64_t)sct * n + mp - 1) / mp);
    for (int mv = 0; mv < 4 * n && mp > 1; mv++) {
        int h = 0, l = 0;
        int64_t tot = 0;
        for (int sct = 0; sct < mp; sct++) {
            tot += Wl[sct];
            if (Wl[sct] > Wl[h]) h = sct;
            if (Wl[sct] < Wl[l]) l = sct;
        }
        if (10 * (int64_t)mp * (Wl[h] - Wl[l]) < tot) break;
        int g = -1;
        if (h > 0) g = h - 1;
        if (h + 1 < mp && (g < 0 || Wl[h + 1] < Wl[g])) g = h + 1;
        if (start[h + 1] == start[h]) break;
        const int c = g < h ? order[start[h]] : order[start[h + 1] - 1];
        const int64_t wc = 2 * Dd(I, 0, c) + I->p[c - 1];
        if (Wl[g] + wc >= Wl[h]) break;
        Wl[g] += wc;
        Wl[h] -= wc;
        if (g < h) start[h]++; else start[h + 1]--;
    }
    /* nearest-neighbour routes, one vehicle per sector */
    char* state = calloc((size_t)n + 1, 1);      /* 0 waiting, 1 dropped, 2 picked */
    int64_t* rdy = calloc((size_t)n + 1, sizeof(int64_t));
    int w = 0;
    off[0] = 0;
    for (int v = 0; v < m; v++) {
        if (v < mp) {
            int64_t t = 0;
            int loc = 0, out = 0;
            const int cnt = start[v + 1] - start[v];
            for (int step = 0; step < 2 * cnt; step++) {
                int bo = -1;
                int64_t bt = 0, bd = 0;
                for (int k = start[v]; k < start[v + 1]; k++) {
                    const int c = order[k];
                    if (state[c] == 2 || (state[c] == 0 && out >= b)) continue;
                    const int pick = state[c] == 1;
                    const int64_t dl = Dd(I, loc, c);
                    int64_t fin = t + dl;
                    if (pick && rdy[c] > fin) fin = rdy[c];
                    const int o = 2 * c + pick;
                    int better = bo < 0;
                    if (!better) {
                        if (fin != bt) better = fin < bt;
                        else if (dl != bd) better = dl < bd;
                        else if ((o & 1) != (bo & 1)) better = (o & 1) < (bo & 1);
                        else better = o < bo;
                    }
                    if (better) { bo = o; bt = fin; bd = dl; }
                }
                const int c = bo >> 1;
                if (bo & 1) { state[c] = 2; out--; }
                else { state[c] = 1; out++; rdy[c] = bt + I->p[c - 1]; }
                t = bt;
                loc = c;
                ops[w++] = bo;
            }
        }
        off[v + 1] = w;
    }
    free(state); free(rdy); free(order); free(start); free(Wl);
    int32_t z;
    uint32_t st;
    oracle_evaluate(I, ops, off, 0, &z, &st, NULL);
    if (st) return -3;
    for (int r = 0; r < refine_rounds; r++) {
        int moved = local_search(I, LS_PICKUP, ops, off, &z, 3);
        moved += local_search(I, LS_RELOCATE, ops, off, &z, 3);
        if (!moved) break;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* BRKGA decoder (Algorithm 2).  keys[0..2n) are op priorities (op index     */
/* 2(c-1)+isPickup); then either m vehicle keys ordering the vehicles for    */
/* tie-breaks (layout 0) or 2n per-op assignment hints (layout 1).           */
/* ------------------------------------------------------------------------ */
/* the vehicle an assignment hint names: floor(m * alpha) in fp64, capped */
static int hint_vehicle(float alpha, int m) {
    double x = (double)alpha * (double)m;
    int h = (int)floor(x);
    if (h > m - 1) h = m - 1;
    if (h < 0) h = 0;
    return h;
}
static const float* g_keys;
static int key_cmp(const void* pa, const void* pb) {
    int a = *(const int*)pa, b = *(const int*)pb;
    if (g_keys[a] < g_keys[b]) return -1;
    if (g_keys[a] > g_keys[b]) return 1;
    return a - b;                                  /* stable: ties by index */
}

int oracle_decode(const oracle_inst* I, const float* keys, int32_t* ops, int32_t* off, int32_t* z_out,
                  int32_t* unsched_out, int64_t* fitness_out) {
    return oracle_decode_l(I, keys, OR_LAYOUT_VKEYS, ops, off, z_out, unsched_out, fitness_out);
}

int oracle_decode_l(const oracle_inst* I, const float* keys, int32_t layout, int32_t* ops, int32_t* off,
                    int32_t* z_out, int32_t* unsched_out, int64_t* fitness_out) {
    const int n = I->n, m = I->m, two_n = 2 * n;
    const int full = (I->flags & OR_LOAD_FULL) != 0;
    int* order = malloc(sizeof(int) * (two_n + 1));
    int* vorder = malloc(sizeof(int) * (m + 1));
    int* rank = malloc(sizeof(int) * (m + 1));
    for (int k = 0; k < two_n; k++) order[k] = k;
    g_keys = keys;
    qsort(order, (size_t)two_n, sizeof(int), key_cmp);                           /* ops by priority */
    for (int v = 0; v < m; v++) vorder[v] = v;
    if (layout == OR_LAYOUT_VKEYS) {
        g_keys = keys + two_n;
        qsort(vorder, (size_t)m, sizeof(int), key_cmp);
    }
    for (int r = 0; r < m; r++) rank[vorder[r]] = r;
    int64_t* t = calloc((size_t)m, sizeof(int64_t));
    int* loc = calloc((size_t)m, sizeof(int));
    int* net = calloc((size_t)m, sizeof(int));
    int* nmin = calloc((size_t)m, sizeof(int));
    int* nmax = calloc((size_t)m, sizeof(int));
    int* load = calloc((size_t)m, sizeof(int));
    int* cnt = calloc((size_t)m, sizeof(int));
    int* seq = malloc(sizeof(int) * (size_t)m * (two_n + 1));
    char* sched = calloc((size_t)two_n + 2, 1);
    int64_t* tdrop = calloc((size_t)n + 1, sizeof(int64_t));
    int64_t sum_load = 0;
    int done = 0;
    for (int pass = 1; pass <= two_n && done < two_n; pass++) {                  /* passes */
        int progress = 0;
        for (int k = 0; k < two_n; k++) {                                       /* ops in priority order */
            int oi = order[k];
            int o = oi + 2, c = o >> 1, pick = o & 1;
            if (sched[o]) continue;
            if (pick && !sched[2 * c]) continue;                                /* a pickup waits for its drop */
            int best = -1;
            int64_t best_arr = 0;
            for (int v = 0; v < m; v++) {
                int ok;
                if (!pick) {
                    if (full) ok = net[v] > -I->Q;                              /* q[v] > 0 */
                    else {
                        int nl = load[v] > -(net[v] - 1) ? load[v] : -(net[v] - 1);
                        int mx = nmax[v] > 0 ? nmax[v] : 0;
                        ok = nl + mx <= I->Q && sum_load - load[v] + nl <= I->R;
                    }
                } else {
                    if (full) ok = net[v] < 0;                                  /* q[v] < k */
                    else ok = load[v] + net[v] + 1 <= I->Q;
                }
                if (!ok) continue;
                int64_t arr = t[v] + Dd(I, loc[v], c);                          /* SelectVehicle */
                if (best < 0 || arr < best_arr || (arr == best_arr && rank[v] < rank[best])) {
                    best = v;
                    best_arr = arr;
                }
            }
            if (best < 0) continue;
            if (layout == OR_LAYOUT_HINTS) {
                /* among the vehicles at the least arrival: the hinted one, then cyclic order */
                const int h = hint_vehicle(keys[two_n + oi], m);
                int bd = m;
                for (int v = 0; v < m; v++) {
                    int ok;
                    if (!pick) {
                        if (full) ok = net[v] > -I->Q;
                        else {
                            int nl = load[v] > -(net[v] - 1) ? load[v] : -(net[v] - 1);
                            int mx = nmax[v] > 0 ? nmax[v] : 0;
                            ok = nl + mx <= I->Q && sum_load - load[v] + nl <= I->R;
                        }
                    } else {
                        if (full) ok = net[v] < 0;
                        else ok = load[v] + net[v] + 1 <= I->Q;
                    }
                    if (!ok || t[v] + Dd(I, loc[v], c) != best_arr) continue;
                    const int dv = ((v - h) % m + m) % m;
                    if (dv < bd) { bd = dv; best = v; }
                }
            }
            int v = best;
            if (!pick) {
                t[v] = best_arr;
                tdrop[c] = best_arr;
                net[v]--;
                if (net[v] < nmin[v]) nmin[v] = net[v];
                int nl = -nmin[v];
                sum_load += nl - load[v];
                load[v] = nl;
            } else {
                int64_t ready = tdrop[c] + I->p[c - 1];
                t[v] = best_arr > ready ? best_arr : ready;
                net[v]++;
                if (net[v] > nmax[v]) nmax[v] = net[v];
            }
            loc[v] = c;
            seq[(size_t)v * (two_n + 1) + cnt[v]++] = o;
            sched[o] = 1;
            done++;
            progress = 1;
        }
        if (!progress) break;
    }
    int64_t z = 0;
    int w = 0;
    off[0] = 0;
    for (int v = 0; v < m; v++) {
        if (cnt[v] > 0) {
            int64_t ret = t[v] + Dd(I, loc[v], 0);                              /* return to the depot */
            if (ret > z) z = ret;
        }
        for (int k = 0; k < cnt[v]; k++) ops[w++] = seq[(size_t)v * (two_n + 1) + k];
        off[v + 1] = w;
    }
    int uns = two_n - done;
    *z_out = (int32_t)z;
    *unsched_out = uns;
    *fitness_out = z + (int64_t)1000000 * uns;     /* Section 4.4.2, infeasibility handling */
    free(order); free(vorder); free(rank); free(t); free(loc); free(net); free(nmin); free(nmax);
    free(load); free(cnt); free(seq); free(sched); free(tdrop);
    return 0;
}

/* ALNS seed encoding (Section 4.4.4): pi_o = (r-1)/L_v; vehicle key v/m
 * (layout 0) or the hint v/m of every op on vehicle v (layout 1), the latter
 * rounded up to the smallest float with m * alpha >= v so that the decoder's
 * floor(m * alpha) names v again. */
static float hint_of(int v, int m) {
    float a = (float)v / (float)m;
    while ((double)a * (double)m < (double)v) a = nextafterf(a, 2.0f);
    return a;
}

void oracle_encode(const oracle_inst* I, const int32_t* ops, const int32_t* off, float* keys) {
    oracle_encode_l(I, ops, off, OR_LAYOUT_VKEYS, keys);
}

void oracle_encode_l(const oracle_inst* I, const int32_t* ops, const int32_t* off, int32_t layout, float* keys) {
    const int n = I->n, m = I->m;
    for (int k = 0; k < (layout == OR_LAYOUT_HINTS ? 4 * n : 2 * n); k++) keys[k] = 0.0f;
    for (int v = 0; v < m; v++) {
        int L = off[v + 1] - off[v];
        for (int r = 0; r < L; r++) {
            keys[ops[off[v] + r] - 2] = (float)r / (float)L;
            if (layout == OR_LAYOUT_HINTS) keys[2 * n + ops[off[v] + r] - 2] = hint_of(v, m);
        }
        if (layout == OR_LAYOUT_VKEYS) keys[2 * n + v] = (float)v / (float)m;
    }
}

/* Construction seeds of the warm start (Section 4.4.4) as decoder
 * chromosomes: every drop before every pickup, both in one customer order;
 * the r-th customer (from 0) gets priority r/(2n) on its drop and (n+r)/(2n)
 * on its pickup, and the decoder builds the schedule.
 *   h = 0 nearest neighbour: the order of the nearest-neighbour tour from the
 *         depot (ties to the smaller id);
 *   h = 1 load-balanced: customers by workload w_c = 2 d(0,c) + p_c (the
 *         workload of Section 4.2.5), largest first; in the hint layout both
 *         ops of c are hinted at the vehicle a greedy least-loaded
 *         assignment in that order gives c (ties to the lower index);
 *   h = 2 shortest processing time: customers by p ascending.
 * Ties go to the smaller id.  The vehicle part is the keys v/m (layout 0) or,
 * for h = 0 and 2, hints naming vehicle 0 (layout 1). */
typedef struct {
    int64_t key;
    int c;
} seed_rank_t;
static int seed_rank_cmp(const void* pa, const void* pb) {
    const seed_rank_t *a = pa, *b = pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return a->c - b->c;
}

void oracle_seed_chromosome(const oracle_inst* I, int32_t h, int32_t layout, float* keys) {
    const int n = I->n, m = I->m;
    int* order = malloc(sizeof(int) * (n + 1));
    int* hv = calloc((size_t)n + 1, sizeof(int));
    if (h == 0) {
        char* vis = calloc((size_t)n + 1, 1);
        int cur = 0;
        for (int r = 0; r < n; r++) {
            int best = -1;
            for (int c = 1; c <= n; c++)
                if (!vis[c] && (best < 0 || Dd(I, cur, c) < Dd(I, cur, best))) best = c;
            vis[best] = 1;
            order[r] = best;
            cur = best;
        }
        free(vis);
    } else {
        seed_rank_t* rk = malloc(sizeof(seed_rank_t) * n);
        for (int c = 1; c <= n; c++) {
            rk[c - 1].c = c;
            rk[c - 1].key = h == 1 ? -(2 * Dd(I, 0, c) + I->p[c - 1]) : (int64_t)I->p[c - 1];
        }
        qsort(rk, (size_t)n, sizeof(seed_rank_t), seed_rank_cmp);
        for (int r = 0; r < n; r++) order[r] = rk[r].c;
        free(rk);
        if (h == 1) {
            int64_t* load = calloc((size_t)m, sizeof(int64_t));
            for (int r = 0; r < n; r++) {
                int v = 0;
                for (int u = 1; u < m; u++)
                    if (load[u] < load[v]) v = u;
                hv[order[r]] = v;
                load[v] += 2 * Dd(I, 0, order[r]) + I->p[order[r] - 1];
            }
            free(load);
        }
    }
    for (int r = 0; r < n; r++) {
        const int c = order[r];
        keys[2 * (c - 1)] = (float)r / (float)(2 * n);
        keys[2 * (c - 1) + 1] = (float)(n + r) / (float)(2 * n);
        if (layout == OR_LAYOUT_HINTS) {
            keys[2 * n + 2 * (c - 1)] = hint_of(hv[c], m);
            keys[2 * n + 2 * (c - 1) + 1] = hint_of(hv[c], m);
        }
    }
    if (layout == OR_LAYOUT_VKEYS)
        for (int v = 0; v < m; v++) keys[2 * n + v] = (float)v / (float)m;
    free(order);
    free(hv);
}

typedef struct {
    int64_t f;
    int idx;
} fit_t;
static int fit_cmp(const void* pa, const void* pb) {
    const fit_t *a = pa, *b = pb;
    if (a->f != b->f) return a->f < b->f ? -1 : 1;
    return a->idx - b->idx;
}

int oracle_brkga_run(const oracle_inst* I, const oracle_brkga_params* P, const int32_t* warm_ops,
                     const int32_t* warm_off, uint64_t seed, float* final_keys, int64_t* trace,
                     int32_t* best_ops, int32_t* best_off, int64_t* best_fitness) {
    const int n = I->n, m = I->m, L = P->layout == OR_LAYOUT_HINTS ? 4 * n : 2 * n + m, pop = P->pop;
    const uint64_t key = stream_key(seed, STREAM_BRKGA), wkey = stream_key(seed, STREAM_WARM);
    const uint64_t per = (uint64_t)L + 2;
    int Ne = (int)floor((double)P->elite_frac * (double)pop);
    int Nm = (int)floor((double)P->mutant_frac * (double)pop);
    if (Ne < 1) Ne = 1;
    if (Ne + Nm > pop) Nm = pop - Ne;
    int Nc = pop - Ne - Nm;
    float* cur = malloc(sizeof(float) * (size_t)pop * L);
    float* nxt = malloc(sizeof(float) * (size_t)pop * L);
    float* base = malloc(sizeof(float) * 4 * L);   /* ALNS encoding, then the three construction seeds */
    fit_t* fit = malloc(sizeof(fit_t) * pop);
    int32_t* dops = malloc(sizeof(int32_t) * 2 * n);
    int32_t* doff = malloc(sizeof(int32_t) * (m + 1));
    /* initial population: warm slots then random keys */
    int warm = warm_ops ? P->warm_slots : 0;
    if (warm > pop) warm = pop;
    if (warm_ops) {
        oracle_encode_l(I, warm_ops, warm_off, P->layout, base);
        for (int h = 0; h < 3; h++) oracle_seed_chromosome(I, h, P->layout, base + (size_t)(h + 1) * L);
    }
    const float top = 1.0f - 1.0f / 16777216.0f;
    const int nvar = P->warm_variants > 0 ? P->warm_variants : 1;
    for (int s = 0; s < pop; s++) {
        float* kk = cur + (size_t)s * L;
        if (s < warm) {
            /* variant 0 is the ALNS encoding itself; with four or more
             * variants the last three perturb the NN, load-balanced and SPT
             * seeds, the others the ALNS encoding */
            int var = s % nvar;
            const float* bs = base + (size_t)(nvar >= 4 && var >= nvar - 3 ? var - (nvar - 3) + 1 : 0) * L;
            for (int g = 0; g < L; g++) {
                if (var == 0) { kk[g] = bs[g]; continue; }
                float u = rng_key(oracle_rng(wkey, (uint64_t)var * L + g));
                float e = (u * 2.0f - 1.0f) * P->eps;                        /* U(-eps, eps) */
                float x = bs[g] + e;
                if (x < 0.0f) x = 0.0f;
                if (x > top) x = top;
                kk[g] = x;
            }
        } else {
            for (int g = 0; g < L; g++) kk[g] = rng_key(oracle_rng(key, (uint64_t)s * per + 2 + g));
        }
    }
    for (int gen = 0; gen < P->generations; gen++) {
        for (int s = 0; s < pop; s++) {
            int32_t z, un;
            int64_t f;
            oracle_decode_l(I, cur + (size_t)s * L, P->layout, dops, doff, &z, &un, &f);
            fit[s].f = f;
            fit[s].idx = s;
        }
        qsort(fit, (size_t)pop, sizeof(fit_t), fit_cmp);
        trace[gen] = fit[0].f;
        if (gen == P->generations - 1) break;
        /* elites, then biased-crossover children, then mutants */
        const uint64_t gbase = (uint64_t)(gen + 1) * (uint64_t)pop;
        for (int k = 0; k < Ne; k++)
            memcpy(nxt + (size_t)k * L, cur + (size_t)fit[k].idx * L, sizeof(float) * L);
        for (int k = 0; k < Nc; k++) {
            int s = Ne + k;
            uint64_t cb = (gbase + (uint64_t)s) * per;
            int e = fit[rng_below(oracle_rng(key, cb + 0), Ne)].idx;
            int o = fit[Ne + rng_below(oracle_rng(key, cb + 1), pop - Ne)].idx;
            for (int g = 0; g < L; g++) {
                float u = rng_key(oracle_rng(key, cb + 2 + g));
                nxt[(size_t)s * L + g] = u < P->rho ? cur[(size_t)e * L + g] : cur[(size_t)o * L + g];
            }
        }
        for (int k = 0; k < Nm; k++) {
            int s = Ne + Nc + k;
            uint64_t cb = (gbase + (uint64_t)s) * per;
            for (int g = 0; g < L; g++) nxt[(size_t)s * L + g] = rng_key(oracle_rng(key, cb + 2 + g));
        }
        float* t = cur; cur = nxt; nxt = t;
    }
    int32_t z, un;
    int64_t f;
    oracle_decode_l(I, cur + (size_t)fit[0].idx * L, P->layout, best_ops, best_off, &z, &un, &f);
    *best_fitness = f;
    if (final_keys) memcpy(final_keys, cur, sizeof(float) * (size_t)pop * L);
    free(cur); free(nxt); free(base); free(fit); free(dops); free(doff);
    return 0;
}
