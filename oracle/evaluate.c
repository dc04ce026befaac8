/*
 * VRP-RPD oracle: instance distances and the candidate evaluator.
 * TEST INFRASTRUCTURE ONLY -- see oracle.h.
 *
 * The evaluator follows the MILP's timing and capacity semantics directly:
 *   drop at arrival (Eq. 7), pickup at departure (Eq. 8), pickup no earlier
 *   than drop + p_c whichever vehicle dropped (Eq. 9), departure >= arrival
 *   (Eq. 10; with a same-vehicle visit this is the wait of Eq. 11), travel
 *   propagation (Eq. 12), return time and makespan (Eqs. 21-23);
 *   capacity: start load (Eq. 13, or the minimal feasible load), bounds
 *   (Eq. 14), update by -drop +pickup (Eqs. 15-16), drop needs a resource
 *   (Eq. 17), pickup needs room (Eq. 18); depot pool: sum of start loads <= R.
 * Operations are processed in a Kahn order: any vehicle whose next op is a
 * drop, or a pickup whose drop is already done, may advance.  Ops that can
 * never be processed form a precedence cycle.
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

void oracle_euc2d(const int32_t* coords, int32_t n_nodes, int32_t* d) {
    for (int i = 0; i < n_nodes; i++)
        for (int j = 0; j < n_nodes; j++) {
            double dx = (double)coords[2 * i] - (double)coords[2 * j];
            double dy = (double)coords[2 * i + 1] - (double)coords[2 * j + 1];
            /* TSPLIB nint: (int)(x + 0.5) */
            d[(int64_t)i * n_nodes + j] = (int32_t)(sqrt(dx * dx + dy * dy) + 0.5);
        }
}

static int64_t D(const oracle_inst* I, int a, int b) {
    return (int64_t)I->d[(int64_t)a * (I->n + 1) + b];
}

int oracle_evaluate(const oracle_inst* I, const int32_t* ops, const int32_t* off,
                    int allow_partial, int32_t* z_out, uint32_t* st_out, int64_t* times) {
    const int n = I->n, m = I->m;
    const int nops = off[m];
    uint32_t st = 0;
    if (times)
        for (int o = 0; o < 2 * n + 2; o++) times[o] = INT64_MIN;
    /* ---- well-formedness ---- */
    if (off[0] != 0 || nops < 0 || nops > 2 * n || (!allow_partial && nops != 2 * n)) st |= OR_MALFORMED;
    for (int v = 0; v < m && !st; v++)
        if (off[v + 1] < off[v]) st |= OR_MALFORMED;
    if (n < 0) return -1;
    char* seen = (char*)calloc((size_t)(2 * n + 2), 1);
    if (!st) {
        for (int k = 0; k < nops; k++) {
            int o = ops[k];
            if (o < 2 || o > 2 * n + 1 || seen[o]) { st |= OR_MALFORMED; break; }
            seen[o] = 1;
        }
        for (int c = 1; c <= n && !st; c++)
            if (seen[2 * c] != seen[2 * c + 1]) st |= OR_MALFORMED;
    }
    if (st) {
        free(seen);
        *z_out = INT32_MAX;
        *st_out = st;
        return 0;
    }
    /* ---- timing: Kahn-order simulation ---- */
    int* pos = (int*)malloc(sizeof(int) * m);
    int* loc = (int*)malloc(sizeof(int) * m);
    int64_t* dep = (int64_t*)malloc(sizeof(int64_t) * m);
    char* dropped = (char*)calloc((size_t)(n + 1), 1);
    int64_t* tdrop = (int64_t*)calloc((size_t)(n + 1), sizeof(int64_t));
    for (int v = 0; v < m; v++) { pos[v] = off[v]; loc[v] = 0; dep[v] = 0; }
    int progress = 1;
    while (progress) {
        progress = 0;
        for (int v = 0; v < m; v++) {
            while (pos[v] < off[v + 1]) {
                int o = ops[pos[v]], c = o >> 1, pick = o & 1;
                if (pick && !dropped[c]) break;         /* Eq. 9 needs T_drop[c] */
                int64_t arr = dep[v] + D(I, loc[v], c); /* Eq. 12 */
                if (!pick) {                            /* Eq. 7 */
                    tdrop[c] = arr;
                    dropped[c] = 1;
                    dep[v] = arr;
                } else {                                /* Eqs. 8-10 */
                    int64_t ready = tdrop[c] + (int64_t)I->p[c - 1];
                    dep[v] = arr > ready ? arr : ready;
                }
                if (times) times[o] = dep[v];
                loc[v] = c;
                pos[v]++;
                progress = 1;
            }
        }
    }
    int64_t z = 0;
    for (int v = 0; v < m; v++) {
        if (pos[v] < off[v + 1]) st |= OR_CYCLE;
        if (off[v + 1] > off[v]) {                      /* Eq. 21; empty route returns at 0 */
            int64_t ret = dep[v] + D(I, loc[v], 0);
            if (ret > z) z = ret;                       /* Eq. 22 */
        }
    }
    /* ---- capacity (Eqs. 13-18) and depot pool ---- */
    int64_t pool = 0;
    for (int v = 0; v < m; v++) {
        int64_t s = 0, smin = 0, smax = 0;
        for (int k = off[v]; k < off[v + 1]; k++) {
            s += (ops[k] & 1) ? 1 : -1;
            if (s < smin) smin = s;
            if (s > smax) smax = s;
        }
        if (I->flags & OR_LOAD_FULL) {
            /* vehicle leaves with Q: stock Q+s must stay in [0,Q] */
            if (smin < -(int64_t)I->Q || smax > 0) st |= OR_VEH_CAP;
            pool += I->Q;
        } else {
            int64_t L = -smin;                          /* smallest load keeping stock >= 0 */
            if (L + smax > I->Q) st |= OR_VEH_CAP;      /* stock L+s <= Q */
            pool += L;
        }
    }
    if (pool > I->R) st |= OR_POOL;
    free(pos); free(loc); free(dep); free(dropped); free(tdrop); free(seen);
    int rc = 0;
    if (st & OR_CYCLE) z = INT32_MAX;
    else if (z > INT32_MAX) { rc = -1; z = INT32_MAX; }
    *z_out = (int32_t)z;
    *st_out = st;
    return rc;
}

typedef struct {
    const oracle_inst* I;
    const int32_t *ops, *off;
    int32_t *z;
    uint32_t* st;
    int32_t lo, hi;
} batch_job;

static void* batch_worker(void* arg) {
    batch_job* j = (batch_job*)arg;
    const int nops = 2 * j->I->n, m1 = j->I->m + 1;
    for (int i = j->lo; i < j->hi; i++)
        oracle_evaluate(j->I, j->ops + (int64_t)i * nops, j->off + (int64_t)i * m1, 0,
                        j->z + i, j->st + i, NULL);
    return NULL;
}

void oracle_evaluate_batch(const oracle_inst* I, int32_t count, const int32_t* ops,
                           const int32_t* off, int32_t* z, uint32_t* status, int32_t threads) {
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    pthread_t tid[256];
    batch_job jobs[256];
    for (int t = 0; t < threads; t++) {
        jobs[t] = (batch_job){I, ops, off, z, status, (int32_t)((int64_t)count * t / threads),
                              (int32_t)((int64_t)count * (t + 1) / threads)};
        if (threads == 1) batch_worker(&jobs[t]);
        else pthread_create(&tid[t], NULL, batch_worker, &jobs[t]);
    }
    if (threads > 1)
        for (int t = 0; t < threads; t++) pthread_join(tid[t], NULL);
}

void oracle_sp_closure(const int32_t* d, int32_t N, int64_t* sp) {
    for (int64_t i = 0; i < (int64_t)N * N; i++) sp[i] = d[i];
    for (int k = 0; k < N; k++)
        for (int i = 0; i < N; i++)
            for (int j = 0; j < N; j++) {
                int64_t via = sp[(int64_t)i * N + k] + sp[(int64_t)k * N + j];
                if (via < sp[(int64_t)i * N + j]) sp[(int64_t)i * N + j] = via;
            }
}

/* Coordination metrics (Section 5.2, "Key Metrics") as counts over the n
 * customers; the percentages are 100 * count / n.
 *   cross: the dropoff and the pickup are on different vehicles.
 *   interleaved: the dropoff vehicle does something else between the
 *     customer's dropoff and its pickup.  On one vehicle: at least one op lies
 *     between the two in the route.  On two vehicles: the dropoff vehicle's
 *     next op exists and is reached (departure after the dropoff plus travel)
 *     before the pickup completes.
 * Returns the evaluator's status.  Counts are -1 where they are undefined:
 * both on a malformed solution, interleaved on a precedence cycle. */
uint32_t oracle_coordination(const oracle_inst* I, const int32_t* ops, const int32_t* off, int32_t* cross,
                             int32_t* interleaved) {
    const int n = I->n, m = I->m;
    int32_t z;
    uint32_t st;
    int64_t* times = (int64_t*)malloc(sizeof(int64_t) * (2 * (size_t)n + 2));
    oracle_evaluate(I, ops, off, 0, &z, &st, times);
    *cross = -1;
    *interleaved = -1;
    if (st & OR_MALFORMED) { free(times); return st; }
    int* veh = (int*)malloc(sizeof(int) * (2 * (size_t)n + 2));
    int* pos = (int*)malloc(sizeof(int) * (2 * (size_t)n + 2));
    for (int v = 0; v < m; v++)
        for (int k = off[v]; k < off[v + 1]; k++) { veh[ops[k]] = v; pos[ops[k]] = k; }
    int nc = 0, ni = 0;
    for (int c = 1; c <= n; c++) {
        const int vd = veh[2 * c], vp = veh[2 * c + 1];
        if (vd != vp) {
            nc++;
            const int nx = pos[2 * c] + 1;
            if (nx < off[vd + 1] && times[2 * c] + D(I, c, ops[nx] >> 1) < times[2 * c + 1]) ni++;
        } else if (pos[2 * c + 1] > pos[2 * c] + 1) {
            ni++;
        }
    }
    *cross = nc;
    if (!(st & OR_CYCLE)) *interleaved = ni;
    free(veh); free(pos); free(times);
    return st;
}
