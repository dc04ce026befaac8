/*
 * VRP-RPD oracle: exhaustive optima used to pin the evaluator.
 * TEST INFRASTRUCTURE ONLY -- see oracle.h.
 *
 *  - oracle_bruteforce: every candidate (all orders of the 2n ops, every
 *    split into m consecutive routes) evaluated by oracle_evaluate; the
 *    minimum over status==0 candidates is the VRP-RPD optimum (Eq. 23).
 *  - oracle_minmax_vrp: the special case of the NP-hardness proof (Section
 *    3.2): with p=0 and capacity >= n, the problem is the min-max VRP; this
 *    enumerates customer orders and splits and never calls the evaluator.
 *  - oracle_held_karp: m=1, p=0 reduces further to the TSP (Held-Karp DP).
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>

typedef struct {
    const oracle_inst* I;
    int32_t* perm;
    int32_t* off;
    int32_t* best_ops;
    int32_t* best_off;
    int64_t best;
    int len;
} bf_state;

static void bf_splits(bf_state* S, int v, int start) {
    const int m = S->I->m;
    if (v == m - 1) {
        S->off[m - 1] = start;
        S->off[m] = S->len;
        int32_t z;
        uint32_t st;
        oracle_evaluate(S->I, S->perm, S->off, 0, &z, &st, NULL);
        if (st == 0 && (S->best < 0 || z < S->best)) {
            S->best = z;
            if (S->best_ops) memcpy(S->best_ops, S->perm, sizeof(int32_t) * S->len);
            if (S->best_off) memcpy(S->best_off, S->off, sizeof(int32_t) * (m + 1));
        }
        return;
    }
    for (int cut = start; cut <= S->len; cut++) {
        S->off[v + 1] = cut;
        bf_splits(S, v + 1, cut);
    }
}

static void bf_perms(bf_state* S, int k) {
    if (k == S->len) {
        S->off[0] = 0;
        bf_splits(S, 0, 0);
        return;
    }
    for (int i = k; i < S->len; i++) {
        int32_t t = S->perm[k]; S->perm[k] = S->perm[i]; S->perm[i] = t;
        bf_perms(S, k + 1);
        t = S->perm[k]; S->perm[k] = S->perm[i]; S->perm[i] = t;
    }
}

int64_t oracle_bruteforce(const oracle_inst* I, int32_t* best_ops, int32_t* best_off) {
    bf_state S;
    S.I = I;
    S.len = 2 * I->n;
    S.perm = (int32_t*)malloc(sizeof(int32_t) * (S.len + 1));
    S.off = (int32_t*)malloc(sizeof(int32_t) * (I->m + 1));
    for (int k = 0; k < S.len; k++) S.perm[k] = 2 + k;
    S.best = -1;
    S.best_ops = best_ops;
    S.best_off = best_off;
    if (I->m == 1) {
        /* single route: splits are trivial */
    }
    bf_perms(&S, 0);
    free(S.perm);
    free(S.off);
    return S.best;
}

/* ---- min-max VRP by enumeration (no evaluator involved) ---- */
typedef struct {
    const int32_t* d;
    int n, m, N;
    int32_t* perm;
    int64_t best;
} mm_state;

static int64_t route_len(const mm_state* S, int a, int b) {
    if (a == b) return 0;
    int64_t L = S->d[S->perm[a]];                       /* d(0, first) */
    for (int k = a + 1; k < b; k++) L += S->d[(int64_t)S->perm[k - 1] * S->N + S->perm[k]];
    L += S->d[(int64_t)S->perm[b - 1] * S->N];          /* d(last, 0) */
    return L;
}

static void mm_splits(mm_state* S, int v, int start, int64_t cur) {
    if (S->best >= 0 && cur >= S->best) return;
    if (v == S->m - 1) {
        int64_t L = route_len(S, start, S->n);
        if (L < cur) L = cur;
        if (S->best < 0 || L < S->best) S->best = L;
        return;
    }
    for (int cut = start; cut <= S->n; cut++) {
        int64_t L = route_len(S, start, cut);
        mm_splits(S, v + 1, cut, L > cur ? L : cur);
    }
}

static void mm_perms(mm_state* S, int k) {
    if (k == S->n) { mm_splits(S, 0, 0, 0); return; }
    for (int i = k; i < S->n; i++) {
        int32_t t = S->perm[k]; S->perm[k] = S->perm[i]; S->perm[i] = t;
        mm_perms(S, k + 1);
        t = S->perm[k]; S->perm[k] = S->perm[i]; S->perm[i] = t;
    }
}

int64_t oracle_minmax_vrp(const int32_t* d, int32_t n, int32_t m) {
    mm_state S = {d, n, m, n + 1, (int32_t*)malloc(sizeof(int32_t) * (n + 1)), -1};
    for (int k = 0; k < n; k++) S.perm[k] = k + 1;
    mm_perms(&S, 0);
    free(S.perm);
    return S.best;
}

int64_t oracle_held_karp(const int32_t* d, int32_t n) {
    const int N = n + 1;
    if (n == 0) return 0;
    const int64_t full = (int64_t)1 << n;
    int64_t* dp = (int64_t*)malloc(sizeof(int64_t) * full * n);
    for (int64_t s = 0; s < full * n; s++) dp[s] = -1;
    for (int j = 0; j < n; j++) dp[((int64_t)1 << j) * n + j] = d[j + 1];   /* 0 -> j+1 */
    for (int64_t s = 1; s < full; s++)
        for (int j = 0; j < n; j++) {
            int64_t cur = dp[s * n + j];
            if (cur < 0) continue;
            for (int k = 0; k < n; k++) {
                if (s & ((int64_t)1 << k)) continue;
                int64_t ns = s | ((int64_t)1 << k);
                int64_t v = cur + d[(int64_t)(j + 1) * N + (k + 1)];
                if (dp[ns * n + k] < 0 || v < dp[ns * n + k]) dp[ns * n + k] = v;
            }
        }
    int64_t best = -1;
    for (int j = 0; j < n; j++) {
        int64_t v = dp[(full - 1) * n + j] + d[(int64_t)(j + 1) * N];
        if (best < 0 || v < best) best = v;
    }
    free(dp);
    return best;
}
