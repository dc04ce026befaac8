// ALNS on the device (Section 4.2, Algorithm 1): the six destroy operators
// of Section 4.2.2 (random, worst, Shaw, cluster, route, critical path), the
// four repair operators of Section 4.2.3 (greedy, regret-2, regret-3,
// regret-m) over the full insertion-delta matrix, simulated-annealing
// acceptance with gated reheat (Section 4.2.4) and adaptive roulette weights
// (Section 4.2.1).
//
// One persistent cooperative launch; a team of CTAs runs one ALNS instance
// and meets at bounded team barriers.  Per iteration:
//   gains   (worst removal only) one skip-walk per customer across the team:
//           the makespan without that customer;
//   begin   rank 0 marks the removed customers (Fisher-Yates, or a block
//           bitonic sort of (key, customer) for the structured operators) and
//           builds W = current solution without them.
// Then one insertion step per removed customer:
//   prep    each CTA stages W in shared memory (op codes packed with their
//           travel-in times).  After a full step, warps walk W from the depot
//           (node times H, makespan) and from every op u (row u of the
//           all-pairs longest-path table LP, and the tail T(u)); after a plain
//           insertion the table is updated in place from the inserted pair
//           instead.  Threads flag "shortcut" gaps, where d(x,c) + d(c,y) <
//           d(x,y) because of the nint rounding;
//   gaps    per-gap vectors (H of the stop before, T of the stop after, the
//           removed leg, stock prefix/suffix extremes), per-(customer, gap)
//           row and column vectors, and sparse tables of the stock prefix;
//           the team then starts the shortcut simulations (schedules with the
//           single shortcut stop added) without waiting for them;
//   matrix  32 x 64 tiles of (dropoff gap, pickup gap) entries for every
//           customer still to insert.  Without shortcut gaps the new makespan
//           is exactly max(z, beta, gamma, delta, epsilon): the old makespan,
//           the longest path through the new drop only, through the new pickup
//           only, through drop -> pickup by the processing edge, and through
//           drop -> route -> pickup (the LP table).  Capacity and pool are O(1)
//           from the prefix/suffix extremes.  Feasible pairs are compacted per
//           CTA and reduced to per-row minima with shared 64-bit atomics.
//           Entries on shortcut gaps come last, from the simulations;
//   select  per-customer argmin of (delta z, delta travel, flat index), then
//           the repair operator's choice across customers; the choice is
//           applied to W.
// Rank 0 ends the iteration: the repaired W is walked and accepted or not,
// the temperature and weights are updated and the next operators are drawn.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cooperative_groups.h>

#include "device_common.cuh"
#include "internal.h"

namespace vrp {

constexpr int NEG = -(1 << 30);               // "unreachable" in the longest-path table
constexpr int UNRES = INT32_MIN;               // ready value not yet published
constexpr int SKIPV = 1 << 28;                 // excluded matrix entry; schedule times stay below 2^27
// Shortcut gaps per greedy step whose simulations run ahead, in the gap phase
// (more than this, rare, are simulated inside the matrix phase instead).
// Per shortcut gap: departures and tails with the drop alone (H1, T1) and with
// the pickup alone (H2, T2), N words each, then z1, h_v1, t_v1, z2, h_v2, t_v2.
constexpr int SC_CAP = 64;
// Each shortcut item is handed out as FB_SPLIT pieces, each taking every
// FB_SPLIT-th block of the row or column: an item's entries are long chains of
// dependent loads, and whole items outlasted the rest of the matrix phase.
constexpr int FB_SPLIT = 8;
constexpr int TR = 32, TC = 64;                // matrix tile rows, cols
constexpr int ALNS_THREADS = 256;
constexpr int ALNS_WARPS = ALNS_THREADS / 32;
constexpr unsigned long long KEY_NONE = ~0ull;
constexpr long long REGRET_INF = 1ll << 40;

struct AlnsCtl {
    int iter, q, nrem, di, rj;
    int z_cur, z_best, z_work;
    unsigned st_work;
    int stagnation, repair_fail, wsel, err;
    int pick_t, pick_row, pick_col;
    unsigned long long wait_ns;       // limit of each spin-wait; one that runs out sets err
    double T, T_init;
    double wd[8], wr[4];
    int sd[8], sr[4], ad[8], ar[4];
    int accepted, improved, new_best, reheats, rejected;
    int z_init;
    // set by the selection when the insertion it applied used no shortcut gap:
    // the next step updates the longest-path table in place of re-walking W.
    // upd: c, x_a, y_a, x_b, y_b (old positions, -1 = depot), adjacent, new
    // positions of D_c and P_c, old length, d(x_a,c), d(c,y_a), d(x_b,c),
    // d(c,y_b), d(c,c), p_c
    int incr;
    int upd[16];
    unsigned long long steps_incr, steps_full;
    unsigned long long phase_ns[7];   // begin, prep, gaps, matrix, select, end, local search (rank 0 wall time)
    // periodic local search: its mode while a candidate's matrix runs (0
    // otherwise), the pass's candidates, the best move so far (customer,
    // makespan, travel, flat gap index, drop route/position, pickup
    // route/position in the solution without the customer)
    int ls, ls_ncand, ls_moved, ls_have, ls_bott, ls_rt;
    int ls_c, ls_bz, ls_a, ls_ia, ls_b, ls_jb;
    int ls_moves, ls_new_best;
    long long ls_travel, ls_bt, ls_bflat;
    int imports;                      // best-of-all solutions this replica took at checkpoints
    // Words that the whole team hits with atomics or polls, each group on a
    // cache line of its own: the CTA that selects an insertion while the
    // others wait reads and writes the state above without meeting their
    // traffic.
    alignas(128) unsigned bar_count;
    alignas(128) unsigned bar_gen;
    alignas(128) int work_counter;
    alignas(128) int walks_done;      // shortcut simulations finished in this greedy step
    alignas(128) int n_short;
    int sum_load;
    alignas(128) unsigned long long entries, fallback_entries;
    unsigned long long pruned;        // tile entries skipped by the bound (counted in entries too)
    unsigned long long tiles, tiles_pruned;  // matrix tiles run, and those with no customer left to score
};

struct AlnsTeam {
    // instance
    int n, m, R, Q, load_full;
    const int* d32;
    const int* p;          // p[0..n]
    // parameters
    double T0, alpha, reheat, r, w_min;
    int stagnation_limit, tau, sigma1, sigma2, sigma3, q_min, q_max, iterations, repair_mask;
    int destroy_mask;        // bit 0 random, 1 worst, 2 Shaw, 3 cluster, 4 route, 5 critical path
    int ls_pickup, ls_relocate;  // local-search periods in iterations (0 = off)
    int replica, nreplicas, sync_every;   // multi-instance: this team's index, team count, checkpoint period
    unsigned* gbar;          // [2] grid barrier over all teams: count, generation
    const AlnsTeam* sib;     // device array of all teams (siblings' best solutions at checkpoints)
    unsigned long long key;  // RNG stream key
    int mode;                // 0 = search, 1 = one-customer matrix dump, 2 = refine the start solution,
                             // 3 = dump_steps repair steps, then mode 1 on the first customer left
    int refine_rounds;       // mode 2: local-search rounds at most
    int dump_c;
    int dump_steps;          // mode 3
    const int* coords;       // device (n+1) x 2 when distances can be recomputed exactly, else null
    // state and scratch (device)
    AlnsCtl* ctl;
    int *cur_ops, *cur_off, *best_ops, *best_off;
    int *W_ops[2], *W_off[2];
    int *rem, *perm;
    int *H, *T, *Ms;
    int *H2, *T2, *Ms2;      // the other copy of each: written by the incremental update, then swapped
    int *S_, *PMINp, *PMAXp, *SMINs, *SMAXs;
    int *spmin, *spmax;      // [LOG][2n]
    int log_levels;
    int *gx, *gy, *gHx, *gTy, *gw, *gsb, *gpmin, *gpmax, *gsmin, *gsmax, *groute, *gpos;
    int *rload;              // start load per route
    int *growc, *gcolc;      // [G][RV], [G][CV]: per-gap constants of the matrix tiles
    int4 *vrow, *vcol;       // [q_max][G]: per (customer, gap) row / column vectors of the matrix
    int2 *vadj;              // [q_max][G]: per (customer, gap) adjacent-pair vector
    unsigned long long* keys;  // [q_max][G]: per drop gap, best (dz, dt, col)
    unsigned long long* rkeys; // [q_max][32]: per drop vehicle, best (dz, dt, row)
    unsigned long long* gmin;  // [q_max][4]: per vehicle group (v mod 4), best (dz, dt) seen so far
    int4* bands;               // [q_max][band_stride]: per 32 gaps, least row x, row w, col x, col w
    int band_stride;
    unsigned char* sc;         // [q_max][G]
    int* slist;                // [q_max * G] entries t * G + g
    int* scix;                 // [q_max][G]: index in slist of a shortcut (customer, gap)
    int* scw;                  // [SC_CAP][scw_stride]: walks of the first SC_CAP shortcut gaps (below)
    int scw_stride;
    int* scpair;               // [SC_CAP][SC_CAP]: makespan with both stops in two shortcut gaps of one customer
    int* trace;
    int* gains;                // [n+1]: removal gain z(cur) - z(cur - c), worst removal
    int* lscand;               // [n+1]: local-search candidates of the current pass
    int4* lsmask;              // [slots]: allowed drop routes, pickup routes, fixed drop gap (-1 any)
    int* dump_delta;
    int* dump_travel;
};

// ---------------------------------------------------------------------------
// shared-memory layout of one CTA
// ---------------------------------------------------------------------------
struct Smem {
    int* sW;        // packed W ops [2n + 4]
    int* sWoff;     // [m + 1]
    int* sp;        // p[0..n]
    int* rdy;       // [warps][n + 1] walk buffers; also the matrix batch vectors and select / begin scratch
    int* rowv;      // [TR][RV]
    int* colv;      // [TC][CV]
    int* misc;      // 64 ints
    unsigned char* flags;  // [n + 1] removed flags / route-start bits
    int* xy;        // coordinates [n + 1][2] (when staged)
};
constexpr int RV = 16, CV = 12;   // row / col vector widths (ints)
constexpr int CB = 8;             // customers per matrix batch
// A tile's batch vectors, row minima and pair list (words), then the list of
// the customers the tile still has to score (up to ACT_CAP of them; with more
// customers waiting, every tile scores every customer).
constexpr int TILE_WORDS = CB * (4 * TC + 8 * TR) + 2 * TR * TC;
constexpr int ACT_CAP = 256;

// Walk buffers (one ready array per warp).  The same words hold a matrix
// tile's batch vectors, row minima and pair list, a shortcut item's
// two walk buffers with its departure and tail arrays, the selection's
// per-customer results (5 words per removed customer) and the removal
// permutation (n words) or a structured destroy's sort keys and per-customer
// facts; no phase needs two of these at once.
__host__ __device__ inline size_t rdy_words(int n) {
    const size_t rw = static_cast<size_t>(((n + 1) + 3) & ~3);
    const size_t walks = static_cast<size_t>(ALNS_WARPS) * rw;
    const size_t fb = 2 * rw + 2 * ((static_cast<size_t>(2 * n) + 3) & ~static_cast<size_t>(3));
    // tile: column and row vectors, adjacent-pair vectors and row minima per
    // customer of a batch, then the compacted pair list (int2 per pair)
    const size_t batch = static_cast<size_t>(TILE_WORDS) + ACT_CAP;
    const size_t sel = 5 * static_cast<size_t>(n) + 8;
    size_t w = walks > batch ? walks : batch;
    w = w > fb ? w : fb;
    w = w > sel ? w : sel;
    w = w > static_cast<size_t>(n) + 4 ? w : static_cast<size_t>(n) + 4;
    // structured destroy: u64 sort keys (a power of two >= n) and five
    // per-customer arrays
    size_t P = 1;
    while (P < static_cast<size_t>(n)) P <<= 1;
    w = w > 2 * P + 5 * rw ? w : 2 * P + 5 * rw;
    return (w + 3) & ~static_cast<size_t>(3);
}

__host__ __device__ inline size_t alns_smem_words(int n, int m, bool with_coords) {
    size_t w = 0;
    w += ((2 * n + 4) + 3) & ~3;
    w += ((m + 1) + 3) & ~3;
    w += ((n + 1) + 3) & ~3;
    w += rdy_words(n);
    w += TR * RV + TC * CV + 64;
    w += ((n + 1 + 3) / 4 + 3) & ~3;
    if (with_coords) w += ((2 * (n + 1)) + 3) & ~3;   // coordinates
    return w;
}

__device__ inline Smem carve(int* base, int n, int m) {
    Smem s;
    int* q = base;
    s.sW = q; q += ((2 * n + 4) + 3) & ~3;
    s.sWoff = q; q += ((m + 1) + 3) & ~3;
    s.sp = q; q += ((n + 1) + 3) & ~3;
    s.rdy = q; q += rdy_words(n);
    s.rowv = q; q += TR * RV;
    s.colv = q; q += TC * CV;
    s.misc = q; q += 64;
    s.flags = reinterpret_cast<unsigned char*>(q);
    q += ((n + 1 + 3) / 4 + 3) & ~3;
    s.xy = q;
    return s;
}

__device__ __forceinline__ int D(const AlnsTeam& t, int a, int b) { return __ldg(t.d32 + a * (t.n + 1) + b); }

// Same value as D: recomputed exactly (EUC_2D) from shared-memory coordinates
// when the instance has small ones, so no L2 round trip sits on the path.
__device__ __forceinline__ int Dx(const AlnsTeam& t, const Smem& s, int a, int b) {
    if (t.coords) return euc2d_small(s.xy[2 * a], s.xy[2 * a + 1], s.xy[2 * b], s.xy[2 * b + 1]);
    return __ldg(t.d32 + a * (t.n + 1) + b);
}

// ---------------------------------------------------------------------------
// team barrier: all CTAs of the team; bounded (about 2 s), sets ctl->err
// ---------------------------------------------------------------------------
__device__ bool team_barrier(AlnsCtl* ctl, int team_blocks, unsigned& gen) {
    __syncthreads();
    if (team_blocks > 1) {
        if (threadIdx.x == 0) {
            volatile unsigned* vgen = &ctl->bar_gen;
            __threadfence();
            const unsigned arrived = atomicAdd(&ctl->bar_count, 1u) + 1u;
            if (arrived == static_cast<unsigned>(team_blocks)) {
                ctl->bar_count = 0u;
                __threadfence();
                atomicExch(&ctl->bar_gen, gen + 1u);
            } else {
                const uint64_t t0 = global_ns();
                while (*vgen == gen) {
                    if (global_ns() - t0 > ctl->wait_ns) {
                        atomicExch(&ctl->err, DEV_TIMEOUT_BARRIER);
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __threadfence();
        }
        gen += 1u;
        __syncthreads();
    }
    return *reinterpret_cast<volatile int*>(&ctl->err) == 0;
}

// The same barrier in two halves, so a CTA can do work that no one waits on
// at the barrier (the shortcut simulations) between arriving and waiting.
__device__ void team_arrive(AlnsCtl* ctl, int team_blocks, unsigned gen) {
    __syncthreads();
    if (team_blocks > 1 && threadIdx.x == 0) {
        __threadfence();
        const unsigned arrived = atomicAdd(&ctl->bar_count, 1u) + 1u;
        if (arrived == static_cast<unsigned>(team_blocks)) {
            ctl->bar_count = 0u;
            __threadfence();
            atomicExch(&ctl->bar_gen, gen + 1u);
        }
    }
}

__device__ bool team_wait(AlnsCtl* ctl, int team_blocks, unsigned& gen) {
    __syncthreads();
    if (team_blocks > 1) {
        if (threadIdx.x == 0) {
            volatile unsigned* vgen = &ctl->bar_gen;
            const uint64_t t0 = global_ns();
            while (*vgen == gen) {
                if (global_ns() - t0 > ctl->wait_ns) {
                    atomicExch(&ctl->err, DEV_TIMEOUT_BARRIER);
                    break;
                }
                __nanosleep(64);
            }
            __threadfence();
        }
        gen += 1u;
        __syncthreads();
    }
    return *reinterpret_cast<volatile int*>(&ctl->err) == 0;
}

// ---------------------------------------------------------------------------
// stage W into shared memory: packed (travel-in << 12 | op)
// ---------------------------------------------------------------------------
__device__ void stage_ops(const AlnsTeam& t, const Smem& s, const int* W, const int* Wo) {
    const int m = t.m;
    for (int i = threadIdx.x; i <= m; i += blockDim.x) s.sWoff[i] = Wo[i];
    __syncthreads();
    const int N = s.sWoff[m];
    // every load of a thread in flight together: its ops and the ops before them
    constexpr int SU = 8;
    for (int k0 = 0; k0 < N; k0 += SU * ALNS_THREADS) {
        int o[SU], pr[SU];
#pragma unroll
        for (int u = 0; u < SU; ++u) {
            const int k = k0 + u * ALNS_THREADS + static_cast<int>(threadIdx.x);
            o[u] = k < N ? W[k] : 0;
            pr[u] = (k < N && k > 0) ? W[k - 1] : 0;
        }
#pragma unroll
        for (int u = 0; u < SU; ++u) {
            const int k = k0 + u * ALNS_THREADS + static_cast<int>(threadIdx.x);
            if (k >= N) break;
            // the op before k on its route: none if k starts a route
            int lo = 0, hi = m;                // find route r with off[r] <= k < off[r+1]
            while (hi - lo > 1) {
                int mid = (lo + hi) >> 1;
                if (s.sWoff[mid] <= k) lo = mid; else hi = mid;
            }
            const int prev = (k == s.sWoff[lo]) ? 0 : (pr[u] >> 1);
            s.sW[k] = (Dx(t, s, prev, o[u] >> 1) << PACK_SHIFT) | o[u];
        }
    }
    __syncthreads();
}

__device__ void stage_W(const AlnsTeam& t, const Smem& s) {
    stage_ops(t, s, t.W_ops[t.ctl->wsel], t.W_off[t.ctl->wsel]);
}

// ---------------------------------------------------------------------------
// walks (one warp; lane r walks route r; m <= 32)
// ---------------------------------------------------------------------------
// From the depot: node times H, stock prefixes, makespan, cycle flag.
__device__ void walk_depot(const AlnsTeam& t, const Smem& s, int* rdy_, bool write_arrays, int* z_out,
                           unsigned* st_out) {
    const int* __restrict__ sW = s.sW;
    const int* __restrict__ spp = s.sp;
    int* const Hh = t.H;

    const int lane = threadIdx.x & 31, m = t.m, n = t.n;
    volatile int* rdy = rdy_;
    for (int c = lane; c <= n; c += 32) rdy[c] = UNRES;
    __syncwarp();
    const bool mine = lane < m;
    int pos = mine ? s.sWoff[lane] : 0, end = mine ? s.sWoff[lane + 1] : 0;
    const int start = pos;
    int dep = 0, last = 0, sv = 0, smin = 0, smax = 0;
    bool walking = mine && pos < end, cyc = false;
    // up to two ops per lane per step, both reads up front (see walk_source)
    bool alive = __any_sync(FULL_MASK, walking);
    while (alive) {
        const bool can1 = walking, can2 = walking && pos + 1 < end;
        const int w1 = can1 ? sW[pos] : 0, w2 = can2 ? sW[pos + 1] : 0;
        const int c1 = (w1 & PACK_MASK) >> 1, c2 = (w2 & PACK_MASK) >> 1;
        const bool k1 = (w1 & 1) != 0, k2 = (w2 & 1) != 0;
        const int r1 = (can1 && k1) ? rdy[c1] : 0;
        const int r2 = (can2 && k2) ? rdy[c2] : 0;
        const bool go1 = can1 && (!k1 || r1 != UNRES);
        const bool go2 = go1 && can2 && (!k2 || r2 != UNRES);
        const int a1 = dep + (w1 >> PACK_SHIFT);
        const int d1 = k1 ? max(a1, r1) : a1;
        const int a2 = d1 + (w2 >> PACK_SHIFT);
        const int d2 = k2 ? max(a2, r2) : a2;
        if (go1) {
            if (!k1) rdy[c1] = a1 + spp[c1];
            if (write_arrays) Hh[pos] = d1;
            sv += k1 ? 1 : -1;
            smin = min(smin, sv);
            smax = max(smax, sv);
            dep = d1;
            last = c1;
        }
        if (go2) {
            if (!k2) rdy[c2] = a2 + spp[c2];
            if (write_arrays) Hh[pos + 1] = d2;
            sv += k2 ? 1 : -1;
            smin = min(smin, sv);
            smax = max(smax, sv);
            dep = d2;
            last = c2;
        }
        pos += (go1 ? 1 : 0) + (go2 ? 1 : 0);
        const bool more = pos < end;
        const unsigned prog = __ballot_sync(FULL_MASK, go1);
        if (walking && more && prog == 0u) cyc = true;
        walking = walking && more && prog != 0u;
        __syncwarp();
        alive = prog != 0u && __any_sync(FULL_MASK, walking);
    }
    if (cyc)
        for (; pos < end; ++pos) {
            const int o = sW[pos] & PACK_MASK;
            if (o & 1) { ++sv; smax = max(smax, sv); } else { --sv; smin = min(smin, sv); }
        }
    int ret = (mine && !cyc && end > start) ? dep + Dx(t, s, last, 0) : 0;
    int load = 0;
    bool bad = false;
    if (mine) {
        if (t.load_full) { bad = smin < -t.Q || smax > 0; load = t.Q; }
        else { bad = -smin + smax > t.Q; load = -smin; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        ret = max(ret, __shfl_xor_sync(FULL_MASK, ret, o));
        load += __shfl_xor_sync(FULL_MASK, load, o);
    }
    const unsigned anycyc = __ballot_sync(FULL_MASK, cyc), anybad = __ballot_sync(FULL_MASK, bad);
    unsigned st = (anycyc ? VRPRPD_CYCLE : 0u) | (anybad ? VRPRPD_VEH_CAP : 0u) | (load > t.R ? VRPRPD_POOL : 0u);
    if (anycyc) ret = 0x7fffffff;
    *z_out = ret;
    *st_out = st;
}

// From op u: row u of LP (NEG where unreachable) and T(u).  Up to two ops per
// lane per step; ready times have one writer (the dropping lane) and are read
// volatile, so a pickup sees "unresolved" (and retries) or the final value,
// and the __syncwarp closing each step makes every write of a step visible in
// the next: a step in which no lane moves means a precedence cycle.
__device__ void walk_source(const AlnsTeam& t, const Smem& s, int* rdy_, int u, int N) {
    const int* __restrict__ sW = s.sW;
    const int* __restrict__ spp = s.sp;

    const int lane = threadIdx.x & 31, m = t.m, n = t.n;
    volatile int* rdy = rdy_;
    for (int c = lane; c <= n; c += 32) rdy[c] = UNRES;
    __syncwarp();
    const bool mine = lane < m;
    int pos = mine ? s.sWoff[lane] : 0;
    const int end = mine ? s.sWoff[lane + 1] : 0;
    int val = NEG, last = 0;
    int* row = t.Ms + static_cast<long long>(u) * N;
    bool walking = mine && pos < end;
    // each step reads both candidate stops and both ready times first; a
    // pickup right behind its own drop waits one step
    bool alive = __any_sync(FULL_MASK, walking);
    while (alive) {
        const bool can1 = walking, can2 = walking && pos + 1 < end;
        const int w1 = can1 ? sW[pos] : 0, w2 = can2 ? sW[pos + 1] : 0;
        const int c1 = (w1 & PACK_MASK) >> 1, c2 = (w2 & PACK_MASK) >> 1;
        const bool k1 = (w1 & 1) != 0, k2 = (w2 & 1) != 0;
        const bool at1 = pos == u, at2 = pos + 1 == u;
        const int r1 = (can1 && k1 && !at1) ? rdy[c1] : 0;
        const int r2 = (can2 && k2 && !at2) ? rdy[c2] : 0;
        const bool go1 = can1 && (!k1 || at1 || r1 != UNRES);
        const bool go2 = go1 && can2 && (!k2 || at2 || r2 != UNRES);
        int v1 = (val == NEG) ? NEG : val + (w1 >> PACK_SHIFT);
        if (k1 && !at1) v1 = max(v1, r1);
        if (at1) v1 = 0;
        int v2 = (v1 == NEG) ? NEG : v1 + (w2 >> PACK_SHIFT);
        if (k2 && !at2) v2 = max(v2, r2);
        if (at2) v2 = 0;
        if (go1) {
            if (!k1) rdy[c1] = (v1 == NEG) ? NEG : v1 + spp[c1];
            row[pos] = v1;
            val = v1;
            last = c1;
        }
        if (go2) {
            if (!k2) rdy[c2] = (v2 == NEG) ? NEG : v2 + spp[c2];
            row[pos + 1] = v2;
            val = v2;
            last = c2;
        }
        pos += (go1 ? 1 : 0) + (go2 ? 1 : 0);
        const bool more = pos < end;
        const unsigned prog = __ballot_sync(FULL_MASK, go1);
        if (walking && more && prog == 0u) atomicExch(&t.ctl->err, DEV_BAD_STATE);
        walking = walking && more && prog != 0u;
        __syncwarp();
        alive = prog != 0u && __any_sync(FULL_MASK, walking);
    }
    int tail = (mine && val != NEG) ? val + Dx(t, s, last, 0) : NEG;
    for (int o = 16; o > 0; o >>= 1) tail = max(tail, __shfl_xor_sync(FULL_MASK, tail, o));
    if (lane == 0) t.T[u] = tail;
}

// Forward simulation of W plus up to two stops, V1 (op code o1) at gap (a, i)
// and V2 (op code o2) at gap (b, j); a < 0 or b < 0 leaves one out, and V1
// goes first when both share a gap.  Returns the makespan (INT32_MAX on a
// precedence cycle); with Hb non-null the departure of every W position goes
// to Hb[pos] and V1's to *hv.  Up to two stops per lane per step (see
// walk_source); the legs next to the new stops are read before the walk.
__device__ int walk_fwd(const AlnsTeam& t, const Smem& s, int* rdy_, int a, int i, int o1, int b, int j, int o2,
                        int* Hb, int* hv) {
    const int* __restrict__ sW = s.sW;
    const int* __restrict__ spp = s.sp;

    const int lane = threadIdx.x & 31, m = t.m;
    volatile int* rdy = rdy_;
    const bool mine = lane < m;
    const int base = mine ? s.sWoff[lane] : 0;
    const int L = mine ? s.sWoff[lane + 1] - base : 0;
    // this lane's stops in route order: (gap g0, op v0, leg in tv0, leg after ta0), then (g1, v1, tv1, ta1)
    int nv = 0, g0 = -1, v0 = 0, g1 = -1, v1 = 0, f0 = 0;
    if (mine) {
        if (lane == a) { g0 = i; v0 = o1; f0 = 1; nv = 1; }
        if (lane == b) {
            if (nv == 0) { g0 = j; v0 = o2; nv = 1; }
            else { g1 = j; v1 = o2; nv = 2; }
        }
    }
    auto cust = [&](int k) { return (sW[base + k] & PACK_MASK) >> 1; };
    int tv0 = 0, ta0 = 0, tv1 = 0, ta1 = 0;
    if (nv >= 1) {
        tv0 = Dx(t, s, g0 > 0 ? cust(g0 - 1) : 0, v0 >> 1);
        if (nv == 2 && g1 == g0) {
            tv1 = Dx(t, s, v0 >> 1, v1 >> 1);
            ta1 = g1 < L ? Dx(t, s, v1 >> 1, cust(g1)) : 0;
        } else {
            ta0 = g0 < L ? Dx(t, s, v0 >> 1, cust(g0)) : 0;
            if (nv == 2) {
                tv1 = Dx(t, s, cust(g1 - 1), v1 >> 1);
                ta1 = g1 < L ? Dx(t, s, v1 >> 1, cust(g1)) : 0;
            }
        }
    }
    int k = 0, vi = 0, dep = 0, loc = 0;
    bool pv = false;                           // the previous stop was a new one
    bool walking = mine && (L > 0 || nv > 0);
    const bool any = walking;
    bool cyc = false;
    // the stop at state (W position kk, new stops done vv), its op and the leg into it
    auto peek = [&](int kk, int vv, bool ppv, bool can, bool& virt, bool& real, int& w, int& op, int& leg) {
        virt = can && vv < nv && kk == (vv == 0 ? g0 : g1);
        real = can && !virt && kk < L;                     // never past the route
        w = real ? sW[base + kk] : 0;
        op = virt ? (vv == 0 ? v0 : v1) : (w & PACK_MASK);
        leg = virt ? (vv == 0 ? tv0 : tv1) : (ppv ? (vv == 1 ? ta0 : ta1) : (w >> PACK_SHIFT));
    };
    // two stops per step: both located and both ready times read first
    bool alive = __any_sync(FULL_MASK, walking);
    while (alive) {
        bool vr1, rl1, vr2, rl2;
        int w1, op1, lg1, w2, op2, lg2;
        peek(k, vi, pv, walking, vr1, rl1, w1, op1, lg1);
        const bool can1 = vr1 || rl1;
        const int kb = k + (rl1 ? 1 : 0), vb = vi + (vr1 ? 1 : 0);
        peek(kb, vb, vr1, can1, vr2, rl2, w2, op2, lg2);
        const bool can2 = vr2 || rl2;
        const int c1 = op1 >> 1, c2 = op2 >> 1;
        const bool p1 = (op1 & 1) != 0, p2 = (op2 & 1) != 0;
        const int r1 = (can1 && p1) ? rdy[c1] : 0;
        const int r2 = (can2 && p2) ? rdy[c2] : 0;
        const bool go1 = can1 && (!p1 || r1 != UNRES);
        const bool go2 = go1 && can2 && (!p2 || r2 != UNRES);
        const int a1 = dep + lg1;
        const int d1 = p1 ? max(a1, r1) : a1;
        const int a2 = d1 + lg2;
        const int d2 = p2 ? max(a2, r2) : a2;
        if (go1) {
            if (!p1) rdy[c1] = a1 + spp[c1];
            if (Hb != nullptr) {
                if (vr1) { if (vi == 0 && f0) *hv = d1; }
                else Hb[base + k] = d1;
            }
            dep = d1;
            loc = c1;
        }
        if (go2) {
            if (!p2) rdy[c2] = a2 + spp[c2];
            if (Hb != nullptr) {
                if (vr2) { if (vb == 0 && f0) *hv = d2; }
                else Hb[base + kb] = d2;
            }
            dep = d2;
            loc = c2;
            k = kb + (rl2 ? 1 : 0);
            vi = vb + (vr2 ? 1 : 0);
            pv = vr2;
        } else if (go1) {
            k = kb;
            vi = vb;
            pv = vr1;
        }
        const bool more = k < L || vi < nv;
        const unsigned prog = __ballot_sync(FULL_MASK, go1);
        if (walking && more && prog == 0u) cyc = true;
        walking = walking && more && prog != 0u;
        __syncwarp();
        alive = prog != 0u && __any_sync(FULL_MASK, walking);
    }
    int ret = (mine && any && !cyc) ? dep + Dx(t, s, loc, 0) : 0;
    for (int o = 16; o > 0; o >>= 1) ret = max(ret, __shfl_xor_sync(FULL_MASK, ret, o));
    const unsigned anycyc = __ballot_sync(FULL_MASK, cyc);
    return anycyc ? 0x7fffffff : ret;
}

// Full simulation of W + D_c at gap (a,i) + P_c at gap (b,j): makespan or
// INT32_MAX on a precedence cycle.
__device__ int walk_insert(const AlnsTeam& t, const Smem& s, int* rdy, int c, int a, int i, int b, int j) {
    const int lane = threadIdx.x & 31, n = t.n;
    for (int q = lane; q <= n; q += 32) rdy[q] = UNRES;
    __syncwarp();
    return walk_fwd(t, s, rdy, a, i, 2 * c, b, j, 2 * c + 1, nullptr, nullptr);
}

// W plus one stop V (op code ov) at gap (a, i), forward: the departure time of
// every W position into Hb[pos] and of V into *hv; returns the makespan
// (INT32_MAX on a precedence cycle).  A pickup V without its drop leaves at
// arrival (its ready time is set to 0): the drop's edge comes with the second
// stop, not here.
__device__ int walk_fwd1(const AlnsTeam& t, const Smem& s, int* rdy, int ov, int a, int i, int* Hb, int* hv) {
    const int lane = threadIdx.x & 31, n = t.n;
    for (int q = lane; q <= n; q += 32) rdy[q] = UNRES;
    __syncwarp();
    if (lane == 0 && (ov & 1)) rdy[ov >> 1] = 0;
    __syncwarp();
    return walk_fwd(t, s, rdy, a, i, ov, -1, 0, 0, Hb, hv);
}

// The same graph backward: the tail of every W position (longest path from its
// departure to the end of the schedule, return leg included) into Tb[pos] and
// V's into *tv.  A drop's tail also takes p plus its pickup's tail; V has no
// partner in this graph.  tp: per-customer pickup tails (n + 1 words).  Up to
// two stops per lane per step, as in the forward walks.
__device__ void walk_bwd1(const AlnsTeam& t, const Smem& s, int* tp_, int ov, int a, int i, int* Tb, int* tv) {
    const int* __restrict__ sW = s.sW;
    const int* __restrict__ spp = s.sp;

    const int lane = threadIdx.x & 31, m = t.m, n = t.n;
    volatile int* tp = tp_;
    for (int q = lane; q <= n; q += 32) tp[q] = UNRES;
    __syncwarp();
    const bool mine = lane < m;
    const int base = mine ? s.sWoff[lane] : 0;
    const int L = mine ? s.sWoff[lane + 1] - base : 0;
    const int gv = (mine && lane == a) ? i : -1;
    const int vc = ov >> 1;
    // legs next to V, read before the walk: V -> the stop after it, the stop before V -> V
    int lv = 0, lb = 0;
    if (gv >= 0) {
        lv = Dx(t, s, vc, gv < L ? (sW[base + gv] & PACK_MASK) >> 1 : 0);
        if (gv > 0) lb = Dx(t, s, (sW[base + gv - 1] & PACK_MASK) >> 1, vc);
    }
    const int lastleg = L > 0 ? Dx(t, s, (sW[base + L - 1] & PACK_MASK) >> 1, 0) : 0;
    const int vret = gv >= 0 ? Dx(t, s, vc, 0) : 0;
    // k: W position still to do (counting down); V sits between positions gv-1 and gv
    int k = L - 1, acc = 0;
    bool vdone = gv < 0, nvn = false, first = true;
    bool walking = mine && (L > 0 || !vdone);
    // the stop at state (kk, done), with "the next stop is V" / "no next stop" flags
    auto peek = [&](int kk, bool done, bool nx, bool fst, bool can, bool& virt, bool& real, int& w, int& c, int& leg) {
        virt = can && !done && kk == gv - 1;
        real = can && !virt && kk >= 0;
        w = real ? sW[base + kk] : 0;
        c = virt ? vc : (w & PACK_MASK) >> 1;
        if (virt) leg = fst ? vret : lv;
        else if (fst) leg = lastleg;
        else if (nx) leg = lb;
        else leg = real ? (sW[base + kk + 1] >> PACK_SHIFT) : 0;
    };
    bool alive = __any_sync(FULL_MASK, walking);
    while (alive) {
        bool vr1, rl1, vr2, rl2;
        int w1, c1, lg1, w2, c2, lg2;
        peek(k, vdone, nvn, first, walking, vr1, rl1, w1, c1, lg1);
        const bool can1 = vr1 || rl1;
        const int kb = k - (rl1 ? 1 : 0);
        const bool db = vdone || vr1;
        peek(kb, db, vr1, false, can1, vr2, rl2, w2, c2, lg2);
        const bool can2 = vr2 || rl2;
        const bool dr1 = rl1 && !(w1 & 1), dr2 = rl2 && !(w2 & 1);
        const int r1 = dr1 ? tp[c1] : 0;
        const int r2 = dr2 ? tp[c2] : 0;
        const bool go1 = can1 && (!dr1 || r1 != UNRES);
        const bool go2 = go1 && can2 && (!dr2 || r2 != UNRES);
        int t1 = lg1 + acc;
        if (dr1) t1 = max(t1, spp[c1] + r1);
        int t2 = lg2 + t1;
        if (dr2) t2 = max(t2, spp[c2] + r2);
        if (go1) {
            if (rl1 && !dr1) tp[c1] = t1;
            if (vr1) *tv = t1;
            else Tb[base + k] = t1;
            acc = t1;
        }
        if (go2) {
            if (rl2 && !dr2) tp[c2] = t2;
            if (vr2) *tv = t2;
            else Tb[base + kb] = t2;
            acc = t2;
            k = kb - (rl2 ? 1 : 0);
            vdone = db || vr2;
            nvn = vr2;
            first = false;
        } else if (go1) {
            k = kb;
            vdone = db;
            nvn = vr1;
            first = false;
        }
        const bool more = k >= 0 || !vdone;
        const unsigned prog = __ballot_sync(FULL_MASK, go1);
        if (walking && more && prog == 0u) atomicExch(&t.ctl->err, DEV_BAD_STATE);
        walking = walking && more && prog != 0u;
        __syncwarp();
        alive = prog != 0u && __any_sync(FULL_MASK, walking);
    }
}

// ---------------------------------------------------------------------------
// capacity helpers (Eqs. 13-18 with the minimal or the full start load)
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool cap_ok(const AlnsTeam& t, int mn, int mx, int& load) {
    if (t.load_full) { load = t.Q; return mn >= -t.Q && mx <= 0; }
    mn = min(mn, 0);
    mx = max(mx, 0);
    load = -mn;
    return load + mx <= t.Q;
}

__device__ __forceinline__ int range_min(const AlnsTeam& t, int lo, int hi, int N) {
    const int len = hi - lo + 1;
    const int l = 31 - __clz(len);
    return min(t.spmin[l * N + lo], t.spmin[l * N + hi - (1 << l) + 1]);
}
__device__ __forceinline__ int range_max(const AlnsTeam& t, int lo, int hi, int N) {
    const int len = hi - lo + 1;
    const int l = 31 - __clz(len);
    return max(t.spmax[l * N + lo], t.spmax[l * N + hi - (1 << l) + 1]);
}

__device__ __forceinline__ unsigned long long pack_key(int dz, int dt, int col) {
    return (static_cast<unsigned long long>(static_cast<unsigned>(dz) ^ 0x80000000u) << 32) |
           (static_cast<unsigned long long>(static_cast<unsigned>(dt + (1 << 19)) & 0xFFFFFu) << 12) |
           static_cast<unsigned long long>(col & 0xFFF);
}

// Capacity + pool of one entry from the per-gap arrays (global memory).
// Returns false when infeasible.
__device__ bool entry_capacity(const AlnsTeam& t, int row, int col, int N) {
    const int a = t.groute[row], i = t.gpos[row], b = t.groute[col], j = t.gpos[col];
    int la = 0, lb = 0;
    const int sumL = t.ctl->sum_load;
    if (a != b) {
        const int mnA = min(min(t.gpmin[row], t.gsb[row] - 1), t.gsmin[row] - 1);
        const int mxA = max(t.gpmax[row], t.gsmax[row] - 1);
        const int mnB = min(t.gpmin[col], t.gsmin[col] + 1);
        const int mxB = max(max(t.gpmax[col], t.gsb[col] + 1), t.gsmax[col] + 1);
        if (!cap_ok(t, mnA, mxA, la) || !cap_ok(t, mnB, mxB, lb)) return false;
        return sumL - t.rload[a] - t.rload[b] + la + lb <= t.R;
    }
    if (j == i) {
        const int mn = min(min(t.gpmin[row], t.gsb[row] - 1), t.gsmin[row]);
        const int mx = max(t.gpmax[row], t.gsmax[row]);
        if (!cap_ok(t, mn, mx, la)) return false;
        return sumL - t.rload[a] + la <= t.R;
    }
    const int lo = t.gy[row], hi = t.gx[col];   // stock prefixes between the two gaps
    const int mn = min(min(min(t.gpmin[row], t.gsb[row] - 1), range_min(t, lo, hi, N) - 1), t.gsmin[col]);
    const int mx = max(max(max(t.gpmax[row], range_max(t, lo, hi, N) - 1), t.S_[hi]), t.gsmax[col]);
    if (!cap_ok(t, mn, mx, la)) return false;
    return sumL - t.rload[a] + la <= t.R;
}

__device__ __forceinline__ int travel_delta(const AlnsTeam& t, const Smem& s, int c, int row, int col) {
    auto locx = [&](int g) { return t.gx[g] >= 0 ? (s.sW[t.gx[g]] & PACK_MASK) >> 1 : 0; };
    auto locy = [&](int g) { return t.gy[g] >= 0 ? (s.sW[t.gy[g]] & PACK_MASK) >> 1 : 0; };
    const int xr = locx(row), yr = locy(row);
    if (t.groute[row] == t.groute[col] && t.gpos[row] == t.gpos[col])
        return Dx(t, s, xr, c) + Dx(t, s, c, c) + Dx(t, s, c, yr) - t.gw[row];
    const int xc = locx(col), yc = locy(col);
    return (Dx(t, s, xr, c) + Dx(t, s, c, yr) - t.gw[row]) + (Dx(t, s, xc, c) + Dx(t, s, c, yc) - t.gw[col]);
}

// ---------------------------------------------------------------------------
// phases
// ---------------------------------------------------------------------------
// Stock prefix arrays of route r from the staged W (one warp): what the walk
// from the depot writes, S_ (stock after each op), its running min / max with
// the start at 0, and the suffix min / max of S_ within the route; the route's
// start load goes to rload[r] and is added to sum_load.
__device__ void scan_route_stock(const AlnsTeam& t, const Smem& s, int r) {
    const int lane = threadIdx.x & 31;
    const int st = s.sWoff[r], en = s.sWoff[r + 1];
    int carry = 0, cmin = 0, cmax = 0;
    for (int base = st; base < en; base += 32) {
        const int k = base + lane;
        const bool in = k < en;
        int v = in ? (((s.sW[k] & PACK_MASK) & 1) ? 1 : -1) : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL_MASK, v, o);
            if (lane >= o) v += y;
        }
        const int sv = carry + v;
        int mn = in ? sv : INT32_MAX, mx = in ? sv : INT32_MIN;
        for (int o = 1; o < 32; o <<= 1) {
            const int y1 = __shfl_up_sync(FULL_MASK, mn, o), y2 = __shfl_up_sync(FULL_MASK, mx, o);
            if (lane >= o) { mn = min(mn, y1); mx = max(mx, y2); }
        }
        mn = min(mn, cmin);
        mx = max(mx, cmax);
        if (in) { t.S_[k] = sv; t.PMINp[k] = mn; t.PMAXp[k] = mx; }
        carry = __shfl_sync(FULL_MASK, sv, 31);
        cmin = __shfl_sync(FULL_MASK, mn, 31);
        cmax = __shfl_sync(FULL_MASK, mx, 31);
    }
    __syncwarp();
    int smn = INT32_MAX, smx = INT32_MIN;
    for (int top = en - 1; top >= st; top -= 32) {
        const int k = top - lane;
        const bool in = k >= st;
        const int sv = in ? t.S_[k] : 0;
        int mn = in ? sv : INT32_MAX, mx = in ? sv : INT32_MIN;
        for (int o = 1; o < 32; o <<= 1) {
            const int y1 = __shfl_up_sync(FULL_MASK, mn, o), y2 = __shfl_up_sync(FULL_MASK, mx, o);
            if (lane >= o) { mn = min(mn, y1); mx = max(mx, y2); }
        }
        mn = min(mn, smn);
        mx = max(mx, smx);
        if (in) { t.SMINs[k] = mn; t.SMAXs[k] = mx; }
        smn = __shfl_sync(FULL_MASK, mn, 31);
        smx = __shfl_sync(FULL_MASK, mx, 31);
    }
    if (lane == 0) {
        const int load = t.load_full ? t.Q : -cmin;
        t.rload[r] = load;
        atomicAdd(&t.ctl->sum_load, load);
    }
}

// After inserting D_c into gap (x_a, y_a) and P_c into gap (x_b, y_b), neither
// a shortcut for c, every path of the old graph survives with at least its old
// length, and a new path meets D_c, or P_c, or both.  With LP the old table,
//     A(u) = LP(u,x_a) + d(x_a,c)                    (reaching D_c)
//     E(u) = max(LP(u,x_b), A(u) + d(c,y_a) + LP(y_a,x_b)) + d(x_b,c)
//     B(v) = d(c,y_b) + LP(y_b,v)                    (leaving P_c)
//     D(v) = max(d(c,y_a) + max(LP(y_a,v), LP(y_a,x_b) + d(x_b,c) + B(v)), p_c + B(v))
//     LP'(u,v) = max(LP(u,v), A(u) + D(v), E(u) + B(v)),
// and the same with the depot's start as u (heads H) and its end as v (tails
// T).  When both stops share one gap, D_c is P_c's only predecessor:
// D(v) = max(d(c,c), p_c) + B(v) and the E term drops.  Unreachable is NEG;
// sums stay clear of overflow by clamping NEG to -2^28 first and mapping every
// negative result back to NEG.  Old positions move right by the new stops
// before them; the new table has stride N + 2 and goes to the second buffers.
constexpr int NEGC = -(1 << 28);

__device__ void phase_update(const AlnsTeam& t, const Smem& s, int rank, int team_blocks) {
    AlnsCtl* ctl = t.ctl;
    const int* up = ctl->upd;
    const int xa = up[2], ya = up[3], xb = up[4], yb = up[5], adj = up[6], Pd = up[7], Pp = up[8];
    const int No = up[9], Nn = No + 2;
    const int dxa = up[10], dya = up[11], dxb = up[12], dyb = up[13], dcc = up[14], pc = up[15];
    const int* Mo = t.Ms;
    int* Mn = t.Ms2;
    auto cl = [](int x) { return x == NEG ? NEGC : x; };
    auto fix = [](int x) { return x < 0 ? NEG : x; };
    const int mcp = max(dcc, pc);
    const int Lyx = (!adj && ya >= 0 && xb >= 0) ? cl(Mo[static_cast<long long>(ya) * No + xb]) : NEGC;
    const int hA = (xa >= 0 ? t.H[xa] : 0) + dxa;
    const int hE = adj ? NEGC : max(xb >= 0 ? t.H[xb] : 0, hA + dya + Lyx) + dxb;
    const int tB = dyb + (yb >= 0 ? t.T[yb] : 0);
    const int tD = adj ? mcp + tB : max(dya + (ya >= 0 ? max(t.T[ya], Lyx + dxb + tB) : 0), pc + tB);
    const int LPdp = adj ? mcp : max(pc, Lyx + dya + dxb);
    if (rank == 0 && threadIdx.x == 0) {
        const int z = ctl->z_work;
        ctl->z_work = max(max(z, hA + tD), hE + tB);
    }
    // new position -> 0 (old op, index in *old), 1 (D_c), 2 (P_c)
    auto kind_of = [&](int k, int* old) {
        if (k == Pd) return 1;
        if (k == Pp) return 2;
        *old = k - (k > Pd ? 1 : 0) - (k > Pp ? 1 : 0);
        return 0;
    };
    constexpr int UR = 16;                     // rows per tile; columns = threads
    int* rowA = s.rowv;                        // [UR] A, E, kind, old index
    int* rowE = rowA + UR;
    int* rowK = rowE + UR;
    int* rowO = rowK + UR;
    const int ntr = (Nn + UR - 1) / UR, ntc = (Nn + ALNS_THREADS - 1) / ALNS_THREADS;
    for (int tile = rank; tile < ntr * ntc; tile += team_blocks) {
        const int r0 = (tile / ntc) * UR, c0 = (tile % ntc) * ALNS_THREADS;
        __syncthreads();                       // the previous tile is done with the row values
        if (threadIdx.x < UR) {
            const int k = r0 + threadIdx.x;
            int kind = 3, u = 0, A = NEGC, E = NEGC;
            if (k < Nn) {
                kind = kind_of(k, &u);
                if (kind == 0) {
                    const long long ro = static_cast<long long>(u) * No;
                    A = xa >= 0 ? cl(Mo[ro + xa]) + dxa : NEGC;
                    E = (adj || xb < 0) ? NEGC : max(cl(Mo[ro + xb]), A + dya + Lyx) + dxb;
                }
                if (c0 == 0)
                    t.T2[k] = kind == 0 ? max(t.T[u], max(A + tD, E + tB)) : (kind == 1 ? tD : tB);
            }
            rowA[threadIdx.x] = A;
            rowE[threadIdx.x] = E;
            rowK[threadIdx.x] = kind;
            rowO[threadIdx.x] = u;
        }
        __syncthreads();
        const int k = c0 + threadIdx.x;
        if (k >= Nn) continue;
        int v = 0;
        const int ck = kind_of(k, &v);
        int B = NEGC, D = NEGC;
        if (ck == 0) {
            B = yb >= 0 ? dyb + cl(Mo[static_cast<long long>(yb) * No + v]) : NEGC;
            D = adj ? mcp + B
                    : max(ya >= 0 ? dya + max(cl(Mo[static_cast<long long>(ya) * No + v]), Lyx + dxb + B) : NEGC,
                          pc + B);
        }
        if (r0 == 0)
            t.H2[k] = ck == 0 ? max(t.H[v], max(hA + D, hE + B)) : (ck == 1 ? hA : (adj ? hA + mcp : max(hE, hA + pc)));
        // all old values of this column first: the stores below may not be
        // ordered ahead of these loads
        int old[UR];
#pragma unroll
        for (int rr = 0; rr < UR; ++rr)
            old[rr] = (ck == 0 && rowK[rr] == 0) ? Mo[static_cast<long long>(rowO[rr]) * No + v] : NEG;
#pragma unroll
        for (int rr = 0; rr < UR; ++rr) {
            const int rk = rowK[rr];
            if (rk == 3) break;
            const int A = rowA[rr], E = rowE[rr];
            int val;
            if (rk == 0) {
                if (ck == 0) val = fix(max(old[rr], max(A + D, E + B)));
                else if (ck == 1) val = fix(A);
                else val = fix(adj ? A + mcp : max(E, A + pc));
            } else if (rk == 1) {
                val = ck == 0 ? fix(D) : (ck == 1 ? 0 : LPdp);
            } else {
                val = ck == 0 ? fix(B) : (ck == 1 ? NEG : 0);
            }
            Mn[static_cast<long long>(r0 + rr) * Nn + k] = val;
        }
    }
}

// The staged solution without customer cx: makespan (INT32_MAX on a cycle).
// The stop after a skipped one is reached from the last kept stop (or the
// depot); a route left empty returns at 0.  One stop per lane per step.
__device__ int walk_skip(const AlnsTeam& t, const Smem& s, int* rdy_, int cx) {
    const int lane = threadIdx.x & 31, m = t.m, n = t.n;
    const int* __restrict__ sW = s.sW;
    const int* __restrict__ spp = s.sp;
    volatile int* rdy = rdy_;
    for (int c = lane; c <= n; c += 32) rdy[c] = UNRES;
    __syncwarp();
    const bool mine = lane < m;
    int pos = mine ? s.sWoff[lane] : 0;
    const int end = mine ? s.sWoff[lane + 1] : 0;
    int dep = 0, loc = 0;
    bool skipped = false, any = false, cyc = false;
    bool walking = mine && pos < end;
    bool alive = __any_sync(FULL_MASK, walking);
    while (alive) {
        const int w = walking ? sW[pos] : 0;
        const int c = (w & PACK_MASK) >> 1;
        const bool pick = (w & 1) != 0, skip = walking && c == cx;
        const int rv = (walking && pick && !skip) ? rdy[c] : 0;
        const bool go = walking && (skip || !pick || rv != UNRES);
        if (go && !skip) {
            const int arr = dep + (skipped ? Dx(t, s, loc, c) : (w >> PACK_SHIFT));
            if (pick) dep = max(arr, rv);
            else { dep = arr; rdy[c] = arr + spp[c]; }
            loc = c;
            any = true;
        }
        if (go) { skipped = skip; ++pos; }
        const bool more = pos < end;
        const unsigned prog = __ballot_sync(FULL_MASK, go);
        if (walking && more && prog == 0u) cyc = true;
        walking = walking && more && prog != 0u;
        __syncwarp();
        alive = prog != 0u && __any_sync(FULL_MASK, walking);
    }
    int ret = (mine && any && !cyc) ? dep + Dx(t, s, loc, 0) : 0;
    for (int o = 16; o > 0; o >>= 1) ret = max(ret, __shfl_xor_sync(FULL_MASK, ret, o));
    const unsigned anycyc = __ballot_sync(FULL_MASK, cyc);
    return anycyc ? 0x7fffffff : ret;
}

// Worst removal's gains (Section 4.2.2): every CTA stages the current
// solution, then one warp per customer c walks it without c; gains[c] =
// z(cur) - z(cur - c).
__device__ __noinline__ void phase_gains(const AlnsTeam& t, const Smem& s, int rank, int team_blocks) {
    stage_ops(t, s, t.cur_ops, t.cur_off);
    const int warp = threadIdx.x >> 5;
    const int team_warps = team_blocks * ALNS_WARPS;
    int* rdy = s.rdy + warp * (((t.n + 1) + 3) & ~3);
    const int z = t.ctl->z_cur;
    for (int c = 1 + rank * ALNS_WARPS + warp; c <= t.n; c += team_warps) {
        const int zc = walk_skip(t, s, rdy, c);
        if ((threadIdx.x & 31) == 0) t.gains[c] = z - zc;
    }
}

__device__ void phase_prep(const AlnsTeam& t, const Smem& s, int rank, int team_blocks, bool incr) {
    AlnsCtl* ctl = t.ctl;
    stage_W(t, s);
    const int N = s.sWoff[t.m];
    const int warp = threadIdx.x >> 5;
    const int team_warps = team_blocks * ALNS_WARPS;
    const int gw = rank * ALNS_WARPS + warp;
    int* rdy = s.rdy + warp * (((t.n + 1) + 3) & ~3);
    if (incr) phase_update(t, s, rank, team_blocks);
    // stock arrays and start loads, route by route (the route loads add up into sum_load)
    for (int r = team_warps - 1 - gw; r < t.m; r += team_warps) scan_route_stock(t, s, r);
    for (int unit = gw; !incr && unit <= N; unit += team_warps) {
        if (unit == 0) {
            int z;
            unsigned st;
            walk_depot(t, s, rdy, true, &z, &st);
            if ((threadIdx.x & 31) == 0) { ctl->z_work = z; ctl->st_work = st; }
        } else {
            walk_source(t, s, rdy, unit - 1, N);
        }
    }
    // shortcut gaps (the rounded legs x->c->y shorter than x->y) and key reset
    // for every customer still to insert; W alone decides them.  The CTAs
    // from the top of the team down take this part: the update's tiles go
    // from rank 0 up, and the first CTAs may hold one tile more than the rest.
    const int G = N + t.m, nrem = ctl->nrem;
    const long long total = static_cast<long long>(nrem) * G;
    const long long tid = static_cast<long long>(team_blocks - 1 - rank) * blockDim.x + threadIdx.x;
    const long long nthr = static_cast<long long>(team_blocks) * blockDim.x;
    for (long long e = tid; e < total; e += nthr) {
        const int ti = static_cast<int>(e / G), g = static_cast<int>(e - static_cast<long long>(ti) * G);
        const int c = t.rem[ti];
        int lo = 0, hi = t.m;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s.sWoff[mid] + mid <= g) lo = mid; else hi = mid;
        }
        const int r = lo, pos = g - (s.sWoff[r] + r), L = s.sWoff[r + 1] - s.sWoff[r];
        const int x = pos > 0 ? (s.sW[s.sWoff[r] + pos - 1] & PACK_MASK) >> 1 : 0;
        const int y = pos < L ? (s.sW[s.sWoff[r] + pos] & PACK_MASK) >> 1 : 0;
        const int w = (L == 0) ? 0 : Dx(t, s, x, y);
        const bool shortcut = Dx(t, s, x, c) + Dx(t, s, c, y) < w;
        t.keys[e] = KEY_NONE;
        if (g < 32) t.rkeys[ti * 32 + g] = KEY_NONE;
        if (g == 0)
            for (int k = 0; k < 4; ++k) t.gmin[ti * 4 + k] = KEY_NONE;
        t.sc[e] = shortcut ? 1 : 0;
        if (shortcut) {
            const int slot = atomicAdd(&ctl->n_short, 1);
            t.slist[slot] = ti * G + g;
            t.scix[e] = slot;
        }
    }
}

__device__ void phase_gaps(const AlnsTeam& t, const Smem& s, int rank, int team_blocks) {
    const int m = t.m, N = s.sWoff[m], G = N + m;
    const long long tid = static_cast<long long>(rank) * blockDim.x + threadIdx.x;
    const long long nthr = static_cast<long long>(team_blocks) * blockDim.x;
    // The phase has three independent parts: the per-gap constants, the
    // per-(customer, gap) vectors and the sparse tables.  The vectors take the
    // CTAs from rank 0 up; the constants and the tables take CTAs from the top
    // of the team down, below the last four (which start the shortcut
    // simulations right after this phase), so that no CTA does two parts.
    const int npg = (G + ALNS_THREADS - 1) / ALNS_THREADS;
    const int rank_pg = ((team_blocks - 5 - rank) % team_blocks + team_blocks) % team_blocks;
    const int rank_sp = ((team_blocks - 5 - npg - rank) % team_blocks + team_blocks) % team_blocks;
    const long long tid_pg = static_cast<long long>(rank_pg) * blockDim.x + threadIdx.x;
    for (long long gg = tid_pg; gg < G; gg += nthr) {
        const int g = static_cast<int>(gg);
        int lo = 0, hi = m;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s.sWoff[mid] + mid <= g) lo = mid; else hi = mid;
        }
        const int r = lo, pos = g - (s.sWoff[r] + r), off = s.sWoff[r], L = s.sWoff[r + 1] - off;
        const int xo = pos > 0 ? off + pos - 1 : -1, yo = pos < L ? off + pos : -1;
        const int x = xo >= 0 ? (s.sW[xo] & PACK_MASK) >> 1 : 0;
        const int y = yo >= 0 ? (s.sW[yo] & PACK_MASK) >> 1 : 0;
        t.gx[g] = xo;
        t.gy[g] = yo;
        t.gHx[g] = xo >= 0 ? t.H[xo] : 0;
        t.gTy[g] = yo >= 0 ? t.T[yo] : 0;
        t.gw[g] = L == 0 ? 0 : Dx(t, s, x, y);
        t.gsb[g] = xo >= 0 ? t.S_[xo] : 0;
        t.gpmin[g] = xo >= 0 ? t.PMINp[xo] : 0;
        t.gpmax[g] = xo >= 0 ? t.PMAXp[xo] : 0;
        t.gsmin[g] = yo >= 0 ? t.SMINs[yo] : (1 << 28);
        t.gsmax[g] = yo >= 0 ? t.SMAXs[yo] : -(1 << 28);
        t.groute[g] = r;
        t.gpos[g] = pos;
        // constants of gap g in the matrix tiles: as a drop gap (row) and as a pickup gap (column)
        const int Hx = xo >= 0 ? t.H[xo] : 0, Ty = yo >= 0 ? t.T[yo] : 0;
        const int sb = xo >= 0 ? t.S_[xo] : 0, pmn = xo >= 0 ? t.PMINp[xo] : 0, pmx = xo >= 0 ? t.PMAXp[xo] : 0;
        const int smn = yo >= 0 ? t.SMINs[yo] : (1 << 28), smx = yo >= 0 ? t.SMAXs[yo] : -(1 << 28);
        const int sumL = t.ctl->sum_load, rl = t.rload[r];
        int la = 0, ladj = 0, lb = 0;
        const bool okA = cap_ok(t, min(min(pmn, sb - 1), smn - 1), max(pmx, smx - 1), la);
        const bool okAdj = cap_ok(t, min(min(pmn, sb - 1), smn), max(pmx, smx), ladj);
        const bool okB = cap_ok(t, min(pmn, smn + 1), max(max(pmx, sb + 1), smx + 1), lb);
        int4* rw4 = reinterpret_cast<int4*>(t.growc + static_cast<long long>(g) * RV);
        rw4[0] = make_int4(Hx, Ty, t.gw[g], okAdj && sumL + ladj - rl <= t.R ? 1 : 0);
        rw4[1] = make_int4(0, 0, okA ? la - rl : 1 << 28, 0);
        rw4[2] = make_int4(r, pos, xo, yo);
        rw4[3] = make_int4(pmn, sb, pmx, 0);
        int4* cw4 = reinterpret_cast<int4*>(t.gcolc + static_cast<long long>(g) * CV);
        cw4[0] = make_int4(0, 0, 0, 0);
        cw4[1] = make_int4(okB ? lb - rl : 1 << 28, r, pos, yo);
        cw4[2] = make_int4(xo, smn, smx, Hx + Ty);
    }
    // per (customer, gap): the matrix vectors
    //   row {max(z, beta) (SKIPV on a shortcut gap), A1 + p_c, E, (dtD + 2^19) << 12}
    //   adj {max(z, adjacent) (SKIPV on a shortcut gap), ((dtAdj + 2^19) << 12) + gap}
    //   col {gamma (SKIPV on a shortcut gap), B1, F, (dtP << 12) + gap}
    // Each warp takes 32 consecutive gaps of one customer (G padded to a
    // multiple of 32), so that it can also reduce, per band of 32 gaps, the
    // least row and column terms (the tiles' lower bounds), and fold the
    // adjacent entries (drop and pickup back to back in one gap, exact here)
    // into the keys before any tile runs.
    {
        AlnsCtl* ctl = t.ctl;
        const int nrem = ctl->nrem, z = ctl->z_work, lsm = ctl->ls;
        const int Gp = (G + 31) & ~31;
        const long long total = static_cast<long long>(nrem) * Gp;
        const int sumL = ctl->sum_load;
        for (long long e0 = tid; e0 < total; e0 += nthr) {
            const int ti = static_cast<int>(e0 / Gp), g = static_cast<int>(e0 - static_cast<long long>(ti) * Gp);
            const long long e = static_cast<long long>(ti) * G + g;
            const bool valid = g < G;
            const int c = t.rem[ti], pc = s.sp[c];
            int4 vr = make_int4(SKIPV, 0, 0, 0), vc = make_int4(SKIPV, 0, 0, 0);
            unsigned long long akey = KEY_NONE;
            int r = 0;
            if (valid) {
                int lo = 0, hi = m;
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (s.sWoff[mid] + mid <= g) lo = mid; else hi = mid;
                }
                r = lo;
                const int pos = g - (s.sWoff[r] + r), off = s.sWoff[r], L = s.sWoff[r + 1] - off;
                const int xo = pos > 0 ? off + pos - 1 : -1, yo = pos < L ? off + pos : -1;
                const int x = xo >= 0 ? (s.sW[xo] & PACK_MASK) >> 1 : 0;
                const int y = yo >= 0 ? (s.sW[yo] & PACK_MASK) >> 1 : 0;
                const int Hx = xo >= 0 ? t.H[xo] : 0, Ty = yo >= 0 ? t.T[yo] : 0;
                const int w = (L == 0) ? 0 : Dx(t, s, x, y);
                const int dxc = Dx(t, s, x, c), dcy = Dx(t, s, c, y), dcc = Dx(t, s, c, c);
                const int delta = dxc + dcy;
                const bool shortcut = delta < w;
                // a local-search slot allows some drop gaps (rows) and pickup gaps
                // (columns) only; the others read as excluded
                bool rok = true, cok = true;
                if (lsm) {
                    const int4 mk = t.lsmask[ti];
                    rok = ((static_cast<unsigned>(mk.x) >> r) & 1u) != 0 && (mk.z < 0 || mk.z == g);
                    cok = ((static_cast<unsigned>(mk.y) >> r) & 1u) != 0;
                }
                vr = make_int4(shortcut || !rok ? SKIPV : max(z, Hx + delta + Ty), Hx + dxc + pc, Hx + delta,
                               static_cast<int>(static_cast<unsigned>(delta - w + (1 << 19)) << 12));
                const int2 va = make_int2(shortcut || !(rok && cok) ? SKIPV : max(z, Hx + dxc + max(dcc, pc) + dcy + Ty),
                                          static_cast<int>((static_cast<unsigned>(dxc + dcc + dcy - w + (1 << 19)) << 12) |
                                                           static_cast<unsigned>(g)));
                vc = make_int4(shortcut || !cok ? SKIPV : Hx + Ty + delta, dcy + Ty, delta + Ty,
                               static_cast<int>((static_cast<unsigned>(delta - w) << 12) + static_cast<unsigned>(g)));
                t.vrow[e] = vr;
                t.vadj[e] = va;
                t.vcol[e] = vc;
                // the adjacent entry of gap g: the stock check of the drop and
                // pickup together at g (the tiles' row constant), then its key
                // in the form the tiles' row minima take
                const int sb = xo >= 0 ? t.S_[xo] : 0, pmn = xo >= 0 ? t.PMINp[xo] : 0, pmx = xo >= 0 ? t.PMAXp[xo] : 0;
                const int smn = yo >= 0 ? t.SMINs[yo] : (1 << 28), smx = yo >= 0 ? t.SMAXs[yo] : -(1 << 28);
                int ladj = 0;
                const bool okAdj = cap_ok(t, min(min(pmn, sb - 1), smn), max(pmx, smx), ladj) &&
                                   sumL + ladj - t.rload[r] <= t.R;
                if (okAdj && va.x < SKIPV)
                    akey = (static_cast<unsigned long long>(static_cast<unsigned>(va.x - z) ^ 0x80000000u) << 32) |
                           static_cast<unsigned>(va.y);
                t.keys[e] = akey;
            }
            // band minima (excluded rows / columns left out), one store per warp
            const unsigned rx = __reduce_min_sync(FULL_MASK, vr.x < SKIPV ? static_cast<unsigned>(vr.x) : 0x7fffffffu);
            const unsigned rw = __reduce_min_sync(FULL_MASK, vr.x < SKIPV ? static_cast<unsigned>(vr.w) : 0xffffffffu);
            const unsigned cx = __reduce_min_sync(FULL_MASK, vc.x < SKIPV ? static_cast<unsigned>(vc.x) : 0x7fffffffu);
            const unsigned cw = __reduce_min_sync(FULL_MASK, vc.x < SKIPV ? static_cast<unsigned>(vc.w) : 0xffffffffu);
            const int lane = threadIdx.x & 31;
            if (lane == 0)
                t.bands[static_cast<long long>(ti) * t.band_stride + (g >> 5)] =
                    make_int4(static_cast<int>(rx), static_cast<int>(rw), static_cast<int>(cx), static_cast<int>(cw));
            // adjacent entries per drop vehicle: the gaps of one warp lie on
            // consecutive routes, each reduced by the whole warp
            const int rlo = static_cast<int>(__reduce_min_sync(FULL_MASK, valid ? static_cast<unsigned>(r) : 0xffffffffu));
            const int rhi = static_cast<int>(__reduce_max_sync(FULL_MASK, valid ? static_cast<unsigned>(r) : 0u));
            const unsigned long long rkey = akey == KEY_NONE ? KEY_NONE : ((akey >> 12) << 12) | static_cast<unsigned>(g);
            for (int rr = rlo; rr <= rhi; ++rr) {
                unsigned long long v = valid && r == rr ? rkey : KEY_NONE;
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long other = __shfl_xor_sync(FULL_MASK, v, o);
                    v = other < v ? other : v;
                }
                if (lane == 0 && v != KEY_NONE) {
                    atomicMin(&t.rkeys[ti * 32 + rr], v);
                    atomicMin(&t.gmin[ti * 4 + (rr & 3)], v >> 12);
                }
            }
        }
    }
    // sparse tables of the stock prefix over op positions.  Every range query
    // lies inside one route, so levels stop at the longest route; each CTA
    // builds a segment of SPB positions from a window reaching 2^top further,
    // all levels in shared memory, min then max.
    constexpr int SPB = 256;
    int lmax = 1;
    for (int r = 0; r < m; ++r) lmax = max(lmax, s.sWoff[r + 1] - s.sWoff[r]);
    int top = 0;
    while ((2 << top) <= lmax) ++top;
    const int nseg = (N + SPB - 1) / SPB;
    int* bufA = s.rdy;
    int* bufB = s.rdy + SPB + (1 << top);
    for (int seg = rank_sp; seg < nseg; seg += team_blocks) {
        const int k0 = seg * SPB;
        const int wn = min(SPB + (1 << top), N - k0);
        for (int pass = 0; pass < 2; ++pass) {
            int* spx = pass ? t.spmax : t.spmin;
            __syncthreads();                   // the buffers are free
            for (int k = threadIdx.x; k < wn; k += blockDim.x) {
                const int v = t.S_[k0 + k];
                bufA[k] = v;
                if (k < SPB) spx[k0 + k] = v;
            }
            __syncthreads();
            int* src = bufA;
            int* dst = bufB;
            for (int l = 1; l <= top; ++l) {
                const int h = 1 << (l - 1);
                const int valid = wn - (1 << l) + 1;
                for (int k = threadIdx.x; k < valid; k += blockDim.x)
                    dst[k] = pass ? max(src[k], src[k + h]) : min(src[k], src[k + h]);
                __syncthreads();
                for (int k = threadIdx.x; k < min(SPB, valid); k += blockDim.x) spx[l * N + k0 + k] = dst[k];
                int* q = src; src = dst; dst = q;
            }
        }
    }
    if (rank == 0 && threadIdx.x == 0) t.ctl->work_counter = 0;
}

// Simulations of the shortcut gaps for the matrix phase: per shortcut gap g of
// customer c the graph with D_c alone at g (forward, backward) and with P_c
// alone at g (forward, backward); per pair of shortcut gaps of one customer (g
// itself twice: the adjacent pair) W with both stops.  One warp per
// simulation, handed out from the last CTA down.  They run between arriving
// at the barrier before the matrix phase and waiting at it, so the tiles of
// the other CTAs proceed meanwhile; every finished simulation is counted in
// walks_done, which the shortcut items wait for.
__device__ int gap_walk_items(const AlnsTeam& t) {
    const int ns = min(t.ctl->n_short, SC_CAP);
    return 4 * ns + ns * ns;
}

__device__ void gap_walks(const AlnsTeam& t, const Smem& s, int rank, int team_blocks) {
    const int m = t.m, N = s.sWoff[m], G = N + m;
    {
        AlnsCtl* ctl = t.ctl;
        const int ns = min(ctl->n_short, SC_CAP);
        const int nmax = (t.scw_stride - 8) / 4;
        const int nitems = 4 * ns + ns * ns;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int team_warps = team_blocks * ALNS_WARPS;
        const int gw = (team_blocks - 1 - rank) * ALNS_WARPS + warp;
        int* rdy = s.rdy + warp * (((t.n + 1) + 3) & ~3);
        auto route_of = [&](int g, int* pos) {
            int lo = 0, hi = m;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (s.sWoff[mid] + mid <= g) lo = mid; else hi = mid;
            }
            *pos = g - (s.sWoff[lo] + lo);
            return lo;
        };
        for (int item = gw; item < nitems; item += team_warps) {
            if (item < 4 * ns) {
                const int e = item >> 2, kind = item & 3;
                const int packed = t.slist[e], ti = packed / G, g = packed - ti * G;
                const int c = t.rem[ti];
                int pos = 0;
                const int r = route_of(g, &pos);
                int* base = t.scw + static_cast<long long>(e) * t.scw_stride;
                int* Hb = base + (kind >> 1) * 2 * nmax;
                int* scal = base + 4 * nmax + (kind >> 1) * 3;
                const int ov = 2 * c + (kind >> 1);
                if ((kind & 1) == 0) {
                    int hv = 0;
                    const int z1 = walk_fwd1(t, s, rdy, ov, r, pos, Hb, &hv);
                    if (lane == r) scal[1] = hv;
                    if (lane == 0) scal[0] = z1;
                } else {
                    int tv = 0;
                    walk_bwd1(t, s, rdy, ov, r, pos, Hb + nmax, &tv);
                    if (lane == r) scal[2] = tv;
                }
            } else {
                const int q = item - 4 * ns, e1 = q / ns, e2 = q - e1 * ns;
                const int p1 = t.slist[e1], p2 = t.slist[e2];
                const int ti = p1 / G;
                if (p2 / G != ti) { if (lane == 0) atomicAdd(&ctl->walks_done, 1); continue; }
                int i1 = 0, i2 = 0;
                const int r1 = route_of(p1 - ti * G, &i1), r2 = route_of(p2 - ti * G, &i2);
                if (r1 == r2 && i2 < i1) {           // the pickup before the drop: never feasible
                    if (lane == 0) atomicAdd(&ctl->walks_done, 1);
                    continue;
                }
                const int zn = walk_insert(t, s, rdy, t.rem[ti], r1, i1, r2, i2);
                if (lane == 0) t.scpair[e1 * SC_CAP + e2] = zn;
            }
            // results visible device-wide, then counted
            __threadfence();
            __syncwarp();
            if (lane == 0) atomicAdd(&ctl->walks_done, 1);
        }
    }
}


// One matrix tile (rows rt*TR.., cols ct*TC..) for every customer still to insert.
//
// Whether a (drop gap, pickup gap) pair can take a customer at all does not
// depend on the customer: every customer moves one unit of the resource, and
// the cycle test and the longest path between the two gaps are properties of
// W.  So each thread first settles its 16 pairs (row tid/8, columns
// tid%8 + 8k) into one register each: the longest-path value LP, or the
// sentinel SKIPV when the pair is excluded (capacity, pool, a cycle, a pickup
// gap before the drop gap on one route).  Per customer an entry is then
//     z' = max(max(z, beta), gamma, A1 + p_c + B1, E + LP + F)
// with the row terms in registers and the column terms one 16-byte shared
// load; excluded pairs and shortcut gaps come out at or above SKIPV and never
// win.  The pair in which both gaps coincide (drop and pickup back to back)
// is the adjacent case, handled once per row.

__device__ void matrix_tile(const AlnsTeam& t, const Smem& s, int rt, int ct, int N, int G) {
    AlnsCtl* ctl = t.ctl;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int r0 = rt * TR, c0 = ct * TC;
    int* rowc = s.rowv;                        // [TR][RV] constants of the drop gaps
    int* colc = s.colv;                        // [TC][CV] constants of the pickup gaps
    const int sumL = ctl->sum_load;
    const bool dump = t.mode == 1;
    const int nrem = ctl->nrem;
    const int z = ctl->z_work;
    // Which customers can this tile change the repair operator's pick for?
    // Every entry of customer c here is at least
    //     (max(least row x, least col x), least row w + least col w)
    // over the tile's rows and columns (the band minima).  The pick needs
    // per customer the best entry (greedy and the local search) and, for
    // regret-2 and regret-3, the makespans of the best two or three drop
    // vehicles.  The best of each vehicle group so far bounds the best entry
    // and those makespans from above; an entry whose drop vehicle already has
    // an entry of no larger makespan cannot change that vehicle's makespan.
    // A customer none of whose entries here can matter is not scored.
    // Regret-m needs every vehicle's best and skips only tiles without an
    // admissible entry.  The tiles' own scores tighten the bounds as they go.
    const bool prune_on = !dump && nrem <= ACT_CAP;
    int* act = s.rdy + TILE_WORDS;             // [ACT_CAP] customers to score
    int* nact = s.misc + 12;
    if (tid == 0) *nact = 0;
    int4 bnd_r = make_int4(0, 0, 0, 0), bnd_c0 = bnd_r, bnd_c1 = make_int4(0, 0, 0x7fffffff, -1);
    unsigned long long gm[4] = {KEY_NONE, KEY_NONE, KEY_NONE, KEY_NONE};
    const bool mine = prune_on && tid < nrem;
    const int kind = ctl->ls ? 0 : ctl->rj;
    // drop vehicles of the tile's rows: the routes of gaps r0 and min(G, r0 + TR) - 1
    auto route_of_gap = [&](int g) {
        int lo = 0, hi = t.m;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s.sWoff[mid] + mid <= g) lo = mid; else hi = mid;
        }
        return lo;
    };
    const int va0 = route_of_gap(r0), va1 = route_of_gap(min(G, r0 + TR) - 1);
    unsigned long long vbest = 0;              // largest best makespan among those vehicles (regret)
    if (mine) {
        const int4* bp = t.bands + static_cast<long long>(tid) * t.band_stride;
        bnd_r = bp[rt];
        bnd_c0 = bp[2 * ct];
        if (2 * ct + 1 < ((G + 31) >> 5)) bnd_c1 = bp[2 * ct + 1];
#pragma unroll
        for (int k = 0; k < 4; ++k) gm[k] = t.gmin[tid * 4 + k];
        if (kind == 1 || kind == 2)
            for (int v = va0; v <= va1; ++v) vbest = max(vbest, t.rkeys[tid * 32 + v] >> 32);
    }
    __syncthreads();                           // the previous tile is done with rowc / colc and the vectors
    for (int e = tid; e < TR * (RV / 4) + TC * (CV / 4); e += blockDim.x) {
        if (e < TR * (RV / 4)) {
            const int rr = e / (RV / 4), q = e - rr * (RV / 4);
            int4 v = make_int4(0, 0, 0, 0);
            if (r0 + rr < G) v = reinterpret_cast<const int4*>(t.growc)[static_cast<long long>(r0 + rr) * (RV / 4) + q];
            else if (q == 2) v.x = -1;         // no such gap: route -1
            reinterpret_cast<int4*>(rowc)[e] = v;
        } else {
            const int e2 = e - TR * (RV / 4);
            const int cc = e2 / (CV / 4), q = e2 - cc * (CV / 4);
            int4 v = make_int4(0, 0, 0, 0);
            if (c0 + cc < G) v = reinterpret_cast<const int4*>(t.gcolc)[static_cast<long long>(c0 + cc) * (CV / 4) + q];
            else if (q == 1) v.y = -1;
            reinterpret_cast<int4*>(colc)[e2] = v;
        }
    }
    if (mine) {
        const int lzz = max(bnd_r.x, min(bnd_c0.z, bnd_c1.z));
        const unsigned llo = static_cast<unsigned>(bnd_r.y) + min(static_cast<unsigned>(bnd_c0.w), static_cast<unsigned>(bnd_c1.w));
        bool keep = lzz < SKIPV;
        if (keep && kind <= 2) {
            const unsigned long long ldz = static_cast<unsigned>(lzz - z) ^ 0x80000000u;
            const unsigned long long u = min(min(gm[0], gm[1]), min(gm[2], gm[3]));
            keep = ((ldz << 20) | (llo >> 12)) <= u;   // may be the best entry
            if (!keep && kind > 0) {
                // the second (regret-2) or third (regret-3) least group makespan
                unsigned long long d[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) d[k] = gm[k] >> 20;
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3 - i; ++j) {
                        const unsigned long long a = min(d[j], d[j + 1]), b = max(d[j], d[j + 1]);
                        d[j] = a;
                        d[j + 1] = b;
                    }
                // may lower a drop vehicle's best makespan that counts
                keep = ldz <= d[kind] && ldz < vbest;
            }
        }
        if (keep) act[atomicAdd(nact, 1)] = tid;
    }
    __syncthreads();
    const int na = prune_on ? *nact : nrem;
    auto cust = [&](int i) { return prune_on ? act[i] : i; };
    // Per customer the vectors of the tile's gaps come from the per-step arrays, CB
    // customers per pair of block barriers, into the walk buffers (unused by tiles):
    //   cols [CB][TC] int4, rows [CB][TR] int4, adj [CB][TR] int2.
    int4* cvec = reinterpret_cast<int4*>(s.rdy);
    int4* rvec = cvec + CB * TC;
    int2* avec = reinterpret_cast<int2*>(rvec + CB * TR);
    auto load_batch = [&](int tb, int nb) {
        for (int it = tid; it < nb * (TR + TC); it += blockDim.x) {
            const int k = it / (TR + TC), slot = it - k * (TR + TC);
            const long long vb = static_cast<long long>(cust(tb + k)) * G;
            if (slot < TR) {
                const int Rr = r0 + slot;
                const bool in = Rr < G;
                rvec[k * TR + slot] = in ? t.vrow[vb + Rr] : make_int4(SKIPV, 0, 0, 0);
                avec[k * TR + slot] = in ? t.vadj[vb + Rr] : make_int2(SKIPV, 0);
            } else {
                const int cc = slot - TR, Cg = c0 + cc;
                cvec[k * TC + cc] = Cg < G ? t.vcol[vb + Cg] : make_int4(SKIPV, 0, 0, Cg);
            }
        }
    };
    // this thread's pairs
    const int r = tid >> 3, cb = tid & 7;
    const int* rk = rowc + r * RV;
    const int ra = rk[8];
    const bool row_ok = ra >= 0;               // all 8 lanes of a row agree; no early exit (shuffles below)
    const int R = r0 + r;
    const unsigned ncols = static_cast<unsigned>(max(0, min(TC / 8, (G - c0 - cb + 7) / 8)));  // this thread's columns < G
    // every entry of the tile counts, scored or not
    const unsigned local_entries = row_ok ? static_cast<unsigned>(nrem) * ncols : 0u;
    const unsigned local_pruned = row_ok ? static_cast<unsigned>(nrem - na) * ncols : 0u;
    auto count_entries = [&]() {
        const unsigned we = __reduce_add_sync(FULL_MASK, local_entries);
        const unsigned wp = __reduce_add_sync(FULL_MASK, local_pruned);
        if ((tid & 31) == 0 && we) atomicAdd(&ctl->entries, static_cast<unsigned long long>(we));
        if ((tid & 31) == 0 && wp) atomicAdd(&ctl->pruned, static_cast<unsigned long long>(wp));
    };
    if (tid == 0) {
        atomicAdd(&ctl->tiles, 1ull);
        if (na == 0) atomicAdd(&ctl->tiles_pruned, 1ull);
    }
    if (na == 0) {                             // no customer left to score: no pair work either
        count_entries();
        return;
    }
    int lpv[TC / 8];
    int diag = -1;                             // column slot of the coinciding gap, if in this thread's set
    // both table reads of every pair first, as predicated loads all in flight
    // together: LP(y_a -> x_b) and the cycle test LP(y_b -> x_a) > NEG; the
    // first batch's vectors load while they are in flight
    int lpl[TC / 8], rcl[TC / 8];
    {
        const int xa = rk[10], ya = rk[11];
#pragma unroll
        for (int kk = 0; kk < TC / 8; ++kk) {
            const int* ck = colc + (cb + 8 * kk) * CV;
            const int rb = ck[5], yb = ck[7], xb = ck[8];
            const bool use = row_ok && rb >= 0;
            const bool okl = use && ya >= 0 && xb >= 0;
            const bool okr = use && ra != rb && yb >= 0 && xa >= 0;
            lpl[kk] = okl ? t.Ms[static_cast<long long>(ya) * N + xb] : NEG;
            rcl[kk] = okr ? t.Ms[static_cast<long long>(yb) * N + xa] : NEG;
        }
    }
    load_batch(0, min(CB, na));
#pragma unroll
    for (int kk = 0; kk < TC / 8; ++kk) {
        const int cc = cb + 8 * kk;
        const int* ck = colc + cc * CV;
        int v = SKIPV;
        const int rb = ck[5];
        if (row_ok && rb >= 0) {
            if (ra == rb) {
                const int ia = rk[9], jb = ck[6];
                if (jb == ia) {
                    diag = cc;
                } else if (jb > ia) {
                    const int lo = rk[11], hi = ck[8];
                    const int mn = min(min(min(rk[12], rk[13] - 1), range_min(t, lo, hi, N) - 1), ck[9]);
                    const int mx = max(max(max(rk[14], range_max(t, lo, hi, N) - 1), t.S_[hi]), ck[10]);
                    int l2 = 0;
                    if (cap_ok(t, mn, mx, l2) && sumL - t.rload[ra] + l2 <= t.R) v = lpl[kk];
                }
            } else {
                const int dLA = rk[6], dLB = ck[4];
                if (rcl[kk] == NEG && dLA < (1 << 27) && dLB < (1 << 27) && sumL + dLA + dLB <= t.R) v = lpl[kk];
            }
        }
        lpv[kk] = v;
    }
    const bool adj_ok = rk[3] != 0;
    if (dump) {
        // every entry of the first customer still to insert written out
        // (parity runs): shortcut entries are left to the shortcut items,
        // excluded pairs read "infeasible"
        for (int tb = 0; tb < min(nrem, 1); tb += CB) {
            const int nb = 1;
            __syncthreads();
            if (tb > 0) load_batch(tb, nb);
            __syncthreads();
            for (int k = 0; k < nb; ++k) {
                const int4 rv = rvec[k * TR + r];
                if (!row_ok) continue;
                const bool scR = rv.x >= SKIPV;
#pragma unroll
                for (int kk = 0; kk < TC / 8; ++kk) {
                    const int cc = cb + 8 * kk, Cg = c0 + cc;
                    const int4 g = cvec[k * TC + cc];
                    if (Cg >= G || scR || g.x >= SKIPV) continue;
                    const long long idx = static_cast<long long>(R) * G + Cg;
                    if (cc == diag) {
                        const int2 a = avec[k * TR + r];
                        t.dump_delta[idx] = adj_ok ? a.x - z : 0x7fffffff;
                        t.dump_travel[idx] = adj_ok ? static_cast<int>(static_cast<unsigned>(a.y) >> 12) - (1 << 19) : 0;
                        continue;
                    }
                    const int zz = max(max(rv.x, g.x), max(rv.y + g.y, rv.z + lpv[kk] + g.z));
                    const unsigned lo = static_cast<unsigned>(rv.w) + static_cast<unsigned>(g.w);
                    const bool ok = lpv[kk] != SKIPV;
                    t.dump_delta[idx] = ok ? zz - z : 0x7fffffff;
                    t.dump_travel[idx] = ok ? static_cast<int>(lo >> 12) - (1 << 19) : 0;
                }
            }
        }
        return;
    }
    // Only part of the pairs survive (a sixth to a third at n = 1000), scattered
    // over the tile.  They are compacted into one row-major list for the whole
    // CTA; per batch the customers share the threads out and each thread takes
    // an equal contiguous share of the list for its customer, keeping a running
    // minimum per row that it folds into the row's slot in shared memory when
    // its row changes; once per batch the row minima go to the global keys.
    unsigned long long* rowbest = reinterpret_cast<unsigned long long*>(avec + CB * TR);   // [CB][TR]
    int2* list = reinterpret_cast<int2*>(rowbest + CB * TR);                                // [TR * TC]
    unsigned fm = 0;
#pragma unroll
    for (int kk = 0; kk < TC / 8; ++kk) fm |= (lpv[kk] != SKIPV ? 1u : 0u) << kk;
    const int cnt = __popc(fm);
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL_MASK, incl, o);
        if ((tid & 31) >= o) incl += y;
    }
    int* wsum = s.misc + 16;                   // [ALNS_WARPS] per-warp totals
    if ((tid & 31) == 31) wsum[warp] = incl;
    __syncthreads();
    int woff = 0, total = 0;
#pragma unroll
    for (int w = 0; w < ALNS_WARPS; ++w) {
        const int v = wsum[w];
        woff += w < warp ? v : 0;
        total += v;
    }
    {
        int at = woff + incl - cnt;
#pragma unroll
        for (int kk = 0; kk < TC / 8; ++kk)
            if ((fm >> kk) & 1u) list[at++] = make_int2(lpv[kk], (r << 8) | (cb + 8 * kk));
    }
    for (int q = tid; q < CB * TR; q += blockDim.x) rowbest[q] = KEY_NONE;
    // a tile with no surviving pair has nothing to compute (the adjacent
    // entries were scored with the gap vectors)
    if (total == 0) {
        count_entries();
        return;
    }
    for (int tb = 0; tb < na; tb += CB) {
        const int nb = min(CB, na - tb);
        __syncthreads();                       // the list and the row slots are ready; the previous batch is flushed
        if (tb > 0) load_batch(tb, nb);
        __syncthreads();
        // the batch's customers split the threads (L each, the rest idle); a
        // thread walks a contiguous share of the list for its customer,
        // keeping the running minimum of its current row, and folds it into
        // the row's slot only when its row changes, so a row's slot sees a
        // few atomics rather than one per pair and customer
        const unsigned long long lim = static_cast<unsigned long long>(SKIPV) << 32;
        const int L = ALNS_THREADS / nb;
        const int k = tid / L, li = tid - k * L;
        if (k < nb) {
            const int qb = static_cast<int>((static_cast<long long>(li) * total) / L);
            const int qe = static_cast<int>((static_cast<long long>(li + 1) * total) / L);
            const int4* cv = cvec + k * TC;
            const int4* rw = rvec + k * TR;
            unsigned long long* rb = rowbest + k * TR;
            int cur = -1;
            int4 rv = make_int4(0, 0, 0, 0);
            unsigned long long best = KEY_NONE;
            for (int q = qb; q < qe; ++q) {
                const int2 le = list[q];
                const int rr = le.y >> 8;
                if (rr != cur) {
                    if (best < lim) atomicMin(&rb[cur], best);
                    rv = rw[rr];
                    best = KEY_NONE;
                    cur = rr;
                }
                const int4 g = cv[le.y & 0xFF];
                const int zz = max(max(rv.x, g.x), max(rv.y + g.y, rv.z + le.x + g.z));
                const unsigned lo = static_cast<unsigned>(rv.w) + static_cast<unsigned>(g.w);
                const unsigned long long key = (static_cast<unsigned long long>(static_cast<unsigned>(zz)) << 32) | lo;
                best = key < best ? key : best;
            }
            if (best < lim) atomicMin(&rb[cur], best);
        }
        __syncthreads();
        // row minima of the batch to the global keys, slots back to empty
        for (int q = tid; q < nb * TR; q += blockDim.x) {
            const unsigned long long b = rowbest[q];
            if (b != KEY_NONE) {
                const int k = q / TR, rr = q - k * TR;
                const int ti = cust(tb + k), Rr = r0 + rr, rra = rowc[rr * RV + 8];
                const unsigned long long key =
                    (static_cast<unsigned long long>(static_cast<unsigned>(static_cast<int>(b >> 32) - z) ^ 0x80000000u) << 32) |
                    (b & 0xFFFFFFFFull);
                atomicMin(&t.keys[static_cast<long long>(ti) * G + Rr], key);
                atomicMin(&t.rkeys[ti * 32 + rra], ((key >> 12) << 12) | static_cast<unsigned long long>(Rr));
                atomicMin(&t.gmin[ti * 4 + (rra & 3)], key >> 12);
                rowbest[q] = KEY_NONE;
            }
        }
    }
    count_entries();
}

// Shortcut item: every entry with one shortcut gap g for customer c (the
// rounded legs x->c->y shorter than x->y, so the old paths through (x,y) do not
// all survive and the tile formula's max(z, ...) is not exact).  As a drop gap
// (as_col = 0) the graph W + D_c at g is simulated once, forward (departures
// H1, makespan z1, D_c's time h_d) and backward (tails T1), by two warps at
// once; then every pickup gap (x_b, y_b) that is not a shortcut for c is exact
// in O(1):
//     z' = max(z1, max(H1(x_b) + d(x_b,c), h_d + p_c) + d(c,y_b) + T1(y_b))
// because each path of W + D_c either survives or gains length.  As a pickup
// gap (as_col = 1) the graph is W + P_c with P_c leaving at arrival; for a
// drop gap (x_a, y_a) with drop time t_d = H2(x_a) + d(x_a,c),
//     z' = max(z2, t_d + d(c,y_a) + T2(y_a), t_d + p_c + T2(P_c)).
// Cycles, the pickup-before-drop order and capacity are the tile's tests.
// Entries whose two gaps are both shortcuts for c (the diagonal of g among
// them) are re-simulated in full, in the item of their drop gap.
__device__ void fallback_item(const AlnsTeam& t, const Smem& s, int item, int N, int G) {
    AlnsCtl* ctl = t.ctl;
    const int piece = item % FB_SPLIT;
    item /= FB_SPLIT;
    const int e = item >> 1, as_col = item & 1;
    const int packed = t.slist[e];
    const int ti = packed / G, g = packed - ti * G;
    if (t.mode == 1 && ti != 0) return;        // a dump writes out the first customer only
    const int c = t.rem[ti];
    const int n = t.n, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rw = ((n + 1) + 3) & ~3;
    // the first SC_CAP shortcut gaps were simulated in the gap phase
    const bool pre = e < SC_CAP;
    const int nmax = (t.scw_stride - 8) / 4;
    const int* pbase = t.scw + static_cast<long long>(pre ? e : 0) * t.scw_stride + as_col * 2 * nmax;
    int* Hs = s.rdy + 2 * rw;                  // [N] departures in W + V (simulated here)
    int* Ts = Hs + ((N + 3) & ~3);             // [N] tails in W + V
    int* sh = s.misc + 8;                      // z1, h_v, t_v
    const int ga = t.groute[g], gi = t.gpos[g];
    const int ov = 2 * c + as_col;
    if (!pre && warp == 0) {
        int hv = 0;
        const int z1 = walk_fwd1(t, s, s.rdy, ov, ga, gi, Hs, &hv);
        if (lane == ga) sh[1] = hv;
        if (lane == 0) sh[0] = z1;
    } else if (!pre && warp == 1) {
        int tv = 0;
        walk_bwd1(t, s, s.rdy + rw, ov, ga, gi, Ts, &tv);
        if (lane == ga) sh[2] = tv;
    }
    __syncthreads();
    const int* Hb = pre ? pbase : Hs;
    const int* Tb = pre ? pbase + nmax : Ts;
    const int* scal = pre ? t.scw + static_cast<long long>(e) * t.scw_stride + 4 * nmax + as_col * 3 : sh;
    const int z1 = scal[0], hv = scal[1], tv = scal[2];
    const int z = ctl->z_work, pc = s.sp[c];
    const long long scrow = static_cast<long long>(ti) * G;
    const bool dump = t.mode == 1;
    unsigned cnt = 0;
    auto loc = [&](int pos) { return pos >= 0 ? (s.sW[pos] & PACK_MASK) >> 1 : 0; };
    // a local-search slot's mask (see the gap phase)
    const int lsm = ctl->ls;
    const int4 mk = lsm ? t.lsmask[ti] : make_int4(-1, -1, -1, 0);
    auto allowed = [&](int row, int col) {
        return ((static_cast<unsigned>(mk.x) >> t.groute[row]) & 1u) != 0 && (mk.z < 0 || mk.z == row) &&
               ((static_cast<unsigned>(mk.y) >> t.groute[col]) & 1u) != 0;
    };
    for (int k = piece * blockDim.x + tid; k < G && z1 != 0x7fffffff; k += FB_SPLIT * blockDim.x) {
        if (k == g || t.sc[scrow + k]) continue;              // both gaps shortcuts: below / elsewhere
        const int row = as_col ? k : g, col = as_col ? g : k;
        if (lsm && !allowed(row, col)) continue;
        const int a = t.groute[row], i = t.gpos[row], b = t.groute[col], j = t.gpos[col];
        const long long idx = static_cast<long long>(row) * G + col;
        if (a == b && j < i) {
            if (dump) { t.dump_delta[idx] = 0x7fffffff; t.dump_travel[idx] = 0; }
            continue;
        }
        const int xa = t.gx[row], yb = t.gy[col];
        const bool cyc = xa >= 0 && yb >= 0 && t.Ms[static_cast<long long>(yb) * N + xa] > NEG;
        const bool ok = !cyc && entry_capacity(t, row, col, N);
        int zn;
        if (!as_col) {
            const int xb = t.gx[col];
            const int arr = (xb >= 0 ? Hb[xb] : 0) + Dx(t, s, loc(xb), c);
            const int dep = max(arr, hv + pc);
            zn = max(z1, dep + Dx(t, s, c, loc(yb)) + (yb >= 0 ? Tb[yb] : 0));
        } else {
            const int ya = t.gy[row];
            const int td = (xa >= 0 ? Hb[xa] : 0) + Dx(t, s, loc(xa), c);
            zn = max(z1, max(td + Dx(t, s, c, loc(ya)) + (ya >= 0 ? Tb[ya] : 0), td + pc + tv));
        }
        ++cnt;
        const int dt = travel_delta(t, s, c, row, col);
        if (dump) {
            t.dump_delta[idx] = ok ? zn - z : 0x7fffffff;
            t.dump_travel[idx] = ok ? dt : 0;
        } else if (ok) {
            const unsigned long long key = pack_key(zn - z, dt, col);
            atomicMin(&t.keys[scrow + row], key);
            atomicMin(&t.rkeys[ti * 32 + a], ((key >> 12) << 12) | static_cast<unsigned long long>(row));
            atomicMin(&t.gmin[ti * 4 + (a & 3)], key >> 12);
        }
    }
    // both gaps shortcuts, from the drop gap's item: full re-simulation, one warp each
    if (!as_col) {
        __syncthreads();                       // Hb / Tb done; walk buffers back to one per warp
        int* rdy = s.rdy + warp * rw;
        for (int k0 = (piece * ALNS_WARPS + warp) * 32; k0 < G; k0 += FB_SPLIT * ALNS_WARPS * 32) {
            const int kl = k0 + lane;
            const bool both = kl < G && (kl == g || t.sc[scrow + kl]);
            unsigned todo = __ballot_sync(FULL_MASK, both);
            while (todo) {
                const int col = k0 + __ffs(todo) - 1;
                todo &= todo - 1;
                if (lsm && !allowed(g, col)) continue;
                const int a = ga, i = gi, b = t.groute[col], j = t.gpos[col];
                const long long idx = static_cast<long long>(g) * G + col;
                if (a == b && j < i) {
                    if (dump && lane == 0) { t.dump_delta[idx] = 0x7fffffff; t.dump_travel[idx] = 0; }
                    continue;
                }
                const bool capok = entry_capacity(t, g, col, N);
                const int e2 = t.scix[scrow + col];
                const int zn = (pre && e2 < SC_CAP) ? t.scpair[e * SC_CAP + e2] : walk_insert(t, s, rdy, c, a, i, b, j);
                const bool ok = capok && zn != 0x7fffffff;
                if (lane == 0) {
                    ++cnt;
                    const int dt = travel_delta(t, s, c, g, col);
                    if (dump) {
                        t.dump_delta[idx] = ok ? zn - z : 0x7fffffff;
                        t.dump_travel[idx] = ok ? dt : 0;
                    } else if (ok) {
                        const unsigned long long key = pack_key(zn - z, dt, col);
                        atomicMin(&t.keys[scrow + g], key);
                        atomicMin(&t.rkeys[ti * 32 + a], ((key >> 12) << 12) | static_cast<unsigned long long>(g));
                        atomicMin(&t.gmin[ti * 4 + (a & 3)], key >> 12);
                    }
                }
            }
        }
    }
    const unsigned wc = __reduce_add_sync(FULL_MASK, cnt);
    if (lane == 0 && wc) atomicAdd(&ctl->fallback_entries, static_cast<unsigned long long>(wc));
}

__device__ void phase_matrix(const AlnsTeam& t, const Smem& s) {
    AlnsCtl* ctl = t.ctl;
    const int N = s.sWoff[t.m], G = N + t.m;
    const int RT = (G + TR - 1) / TR, CT = (G + TC - 1) / TC;
    const int tiles = RT * CT;
    // The shortcut items go out first: each scores a whole row or column of
    // G entries, far more work than a tile, so at the end of the phase they
    // would leave most of the team waiting; their simulations are done by the
    // time the phase starts (the team barrier before it waits for every walk).
    const int nfb = 2 * ctl->n_short * FB_SPLIT;
    const int total = tiles + nfb;
    const int nwalks = gap_walk_items(t);
    bool walks_seen = false;
    int* slot = s.misc;
    // local search: tiles that hold no allowed entry are skipped (pickup
    // repositioning: one row of tiles; relocation: tiles whose rows and
    // columns share no route)
    const int lsm = ctl->ls, ls_rt = ctl->ls_rt;
    auto ls_skip = [&](int rt, int ct) {
        if (lsm == 1) return rt != ls_rt;
        if (lsm == 2) {
            const int r0 = rt * TR, r1 = min(G, r0 + TR) - 1, c0 = ct * TC, c1 = min(G, c0 + TC) - 1;
            return t.groute[r1] < t.groute[c0] || t.groute[c1] < t.groute[r0];
        }
        return false;
    };
    // Tiles go out by their distance d = |ct - rt/2| from the diagonal (the
    // column tile that holds the row band's own gaps): the entries near it
    // (drop and pickup on one route or on neighbouring ones) are where a
    // customer's best insertion usually lies, so their scores tighten the
    // bounds before the far tiles are reached.  Per d, the tiles left of the
    // diagonal (ct = rt/2 - d, rt = 2d..RT-1), then those right of it
    // (ct = rt/2 + d, rt = 0..2(CT-d)-1).
    auto tile_of = [&](int item, int* prt, int* pct) {
        if (item < RT) { *prt = item; *pct = item >> 1; return; }
        item -= RT;
        for (int d = 1; d < CT; ++d) {
            const int nl = max(0, RT - 2 * d), nr = max(0, min(RT, 2 * (CT - d)));
            if (item < nl) { *prt = 2 * d + item; *pct = (*prt >> 1) - d; return; }
            item -= nl;
            if (item < nr) { *prt = item; *pct = (item >> 1) + d; return; }
            item -= nr;
        }
        *prt = -1;                             // not reached: the counts add up to RT * CT
        *pct = -1;
    };
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) slot[0] = atomicAdd(&ctl->work_counter, 1);
        __syncthreads();
        const int item = slot[0];
        if (item >= total) break;
        if (item >= nfb) {
            int rt = 0, ct = 0;
            tile_of(item - nfb, &rt, &ct);
            if (rt >= 0 && !ls_skip(rt, ct)) matrix_tile(t, s, rt, ct, N, G);
        } else {
            if (!walks_seen) {
                // the shortcut simulations, still running in other CTAs, must be done (bounded wait)
                if (threadIdx.x == 0) {
                    volatile int* wd = &ctl->walks_done;
                    const uint64_t t0 = global_ns();
                    while (*wd < nwalks) {
                        if (global_ns() - t0 > ctl->wait_ns) {
                            atomicExch(&ctl->err, DEV_TIMEOUT_BARRIER);
                            break;
                        }
                        __nanosleep(256);
                    }
                    __threadfence();
                }
                __syncthreads();
                walks_seen = true;
            }
            fallback_item(t, s, item, N, G);
        }
    }
}

// Insert customer c into the staged solution (s.sW, s.sWoff): its drop at
// position ia of route a, its pickup at position jb of route b (positions in
// the staged solution; on one route jb >= ia and the pickup follows the drop).
// Writes Wn / Won; all threads of the block, element-parallel: old op i of
// route v moves right by the insertions that precede it.
__device__ void insert_staged(const AlnsTeam& t, const Smem& s, int c, int a, int ia, int b, int jb, int* Wn,
                              int* Won) {
    const int m = t.m, N = s.sWoff[m];
    for (int p = threadIdx.x; p < N; p += blockDim.x) {
        int lo = 0, hi = m;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s.sWoff[mid] <= p) lo = mid; else hi = mid;
        }
        const int v = lo, i = p - s.sWoff[v];
        const int shift = (a < v ? 1 : 0) + (b < v ? 1 : 0) + (v == a && i >= ia ? 1 : 0) + (v == b && i >= jb ? 1 : 0);
        Wn[p + shift] = s.sW[p] & PACK_MASK;
    }
    if (threadIdx.x == 0) {
        const int base_a = s.sWoff[a] + (b < a ? 1 : 0);
        Wn[base_a + ia] = 2 * c;
        const int base_b = s.sWoff[b] + (a < b ? 1 : 0);
        Wn[base_b + jb + (a == b ? 1 : 0)] = 2 * c + 1;
    }
    if (threadIdx.x <= m) {
        const int v = threadIdx.x;
        Won[v] = s.sWoff[v] + (a < v ? 1 : 0) + (b < v ? 1 : 0);
    }
}

// Rank 0: per-customer argmin, greedy / regret-k choice, apply to W.
__device__ void phase_select(const AlnsTeam& t, const Smem& s) {
    AlnsCtl* ctl = t.ctl;
    const int m = t.m, N = s.sWoff[m], G = N + m, nrem = ctl->nrem;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // per-customer results in the (now free) walk buffers
    unsigned long long* bestv = reinterpret_cast<unsigned long long*>(s.rdy);       // [nrem] (dz,dt)<<12 | row
    long long* regret = reinterpret_cast<long long*>(s.rdy) + nrem;                // [nrem]
    // the column of a customer's best entry, read from its row key (needed on
    // ties of (dz, dt) between customers and for the one picked)
    int* colv = reinterpret_cast<int*>(regret + nrem);                              // [nrem]
    auto colof = [&](int ti) { return colv[ti]; };
    // A warp takes customers warp, warp + 8, ... four at a time, with the
    // route keys of all four loaded before any is reduced.
    constexpr int SU = 4;
    for (int t0 = warp; t0 < nrem; t0 += SU * ALNS_WARPS) {
        unsigned long long rks[SU];
#pragma unroll
        for (int u = 0; u < SU; ++u) {
            const int ti = t0 + u * ALNS_WARPS;
            rks[u] = (ti < nrem && lane < m) ? t.rkeys[ti * 32 + lane] : KEY_NONE;
        }
#pragma unroll
        for (int u = 0; u < SU; ++u) {
            const int ti = t0 + u * ALNS_WARPS;
            if (ti >= nrem) break;
            // best per drop vehicle (the regret-2 options) and overall, from the route keys
            const unsigned long long rk = rks[u];
            unsigned long long bv = rk;
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long other = __shfl_xor_sync(FULL_MASK, bv, o);
                bv = other < bv ? other : bv;
            }
            // regret-k over the per-vehicle options: the sum over the k best of
            // (c_i - c_1), options past the m there are counting as REGRET_INF;
            // k = 2, 3 or m for repair operators 1, 2, 3 (greedy needs none of it)
            const int rj = ctl->rj;
            long long reg = 0;
            if (rj != 0) {
                const long long cvl = (lane < m && rk != KEY_NONE)
                                          ? static_cast<long long>(static_cast<int>(static_cast<unsigned>(rk >> 32) ^ 0x80000000u))
                                          : REGRET_INF;
                // the least option (with its lane) and the least of the others, by
                // two warp min-reductions of (option + 2^31) << 6 | lane
                const unsigned long long key1 = (static_cast<unsigned long long>(cvl + (1ll << 31)) << 6) |
                                                static_cast<unsigned long long>(lane);
                unsigned long long k1 = key1;
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long other = __shfl_xor_sync(FULL_MASK, k1, o);
                    k1 = other < k1 ? other : k1;
                }
                unsigned long long k2 = (static_cast<int>(k1 & 63u) == lane) ? ~0ull : key1;
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long other = __shfl_xor_sync(FULL_MASK, k2, o);
                    k2 = other < k2 ? other : k2;
                }
                const long long c1 = static_cast<long long>(k1 >> 6) - (1ll << 31);
                const long long c2 = static_cast<long long>(k2 >> 6) - (1ll << 31);
                if (rj == 1) {
                    reg = c2 - c1;
                } else {
                    const int kreg = rj == 2 ? 3 : m;
                    int rnk = 0;
                    for (int v = 0; v < m; ++v) {
                        const long long cu = __shfl_sync(FULL_MASK, cvl, v);
                        if (cu < cvl || (cu == cvl && v < lane)) ++rnk;
                    }
                    long long term = (lane < m && rnk < kreg) ? cvl - c1 : 0;
                    for (int o = 16; o > 0; o >>= 1) term += __shfl_xor_sync(FULL_MASK, term, o);
                    if (kreg > m) term += static_cast<long long>(kreg - m) * (REGRET_INF - c1);
                    reg = term;
                }
            }
            if (lane == 0) {
                bestv[ti] = bv;
                regret[ti] = reg;
            }
        }
        // the best entries' columns, the four loads in flight together
        __syncwarp();
        if (lane < SU) {
            const int ti = t0 + lane * ALNS_WARPS;
            if (ti < nrem) {
                const unsigned long long bv = bestv[ti];
                colv[ti] = bv == KEY_NONE ? 0 : static_cast<int>(t.keys[static_cast<long long>(ti) * G + (bv & 0xFFF)] & 0xFFF);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int pick = -1;
        bool fail = false;
        for (int ti = 0; ti < nrem; ++ti) {
            if (bestv[ti] == KEY_NONE) { fail = true; break; }
            if (pick < 0) { pick = ti; continue; }
            if (ctl->rj == 0) {
                // greedy: (dz, dt), then flat index row*G + col; ties to the smaller customer id
                const unsigned long long pa = bestv[ti] >> 12, pb = bestv[pick] >> 12;
                if (pa != pb) { if (pa < pb) pick = ti; }
                else {
                    const long long fa = static_cast<long long>(bestv[ti] & 0xFFF) * G + colof(ti);
                    const long long fb = static_cast<long long>(bestv[pick] & 0xFFF) * G + colof(pick);
                    if (fa < fb) pick = ti;
                }
            } else {
                if (regret[ti] > regret[pick]) pick = ti;
            }
        }
        int* sel = s.misc + 24;                // fail, customer slot, row, column
        sel[0] = (fail || pick < 0) ? 1 : 0;
        if (fail || pick < 0) {
            ctl->repair_fail = 1;
        } else {
            sel[1] = pick;
            sel[2] = static_cast<int>(bestv[pick] & 0xFFF);
            sel[3] = colof(pick);
            ctl->pick_t = sel[1];
            ctl->pick_row = sel[2];
            ctl->pick_col = sel[3];
        }
    }
    __syncthreads();
    const int* sel = s.misc + 24;
    if (sel[0]) return;
    // apply to the other W buffer; every load the step needs is issued first
    const int pick = sel[1], row = sel[2], col = sel[3];
    const int c = t.rem[pick];
    const int a = t.groute[row], ia = t.gpos[row], b = t.groute[col], jb = t.gpos[col];
    const long long scb = static_cast<long long>(pick) * G;
    int xa = 0, ya = 0, xb = 0, yb = 0;
    bool shortcut = false;
    if (threadIdx.x == 0) {
        shortcut = t.sc[scb + row] != 0 || t.sc[scb + col] != 0;
        xa = t.gx[row]; ya = t.gy[row]; xb = t.gx[col]; yb = t.gy[col];
    }
    // the customers still to insert without the inserted one, order kept (in
    // registers for the first blockDim.x of them)
    const int k0 = threadIdx.x;
    const int remv = k0 + 1 < nrem ? t.rem[k0 + (k0 >= pick ? 1 : 0)] : 0;
    insert_staged(t, s, c, a, ia, b, jb, t.W_ops[ctl->wsel ^ 1], t.W_off[ctl->wsel ^ 1]);
    if (threadIdx.x == 0) {
        // the next step updates the longest-path table incrementally unless a
        // gap of this insertion was a shortcut for c
        int* up = ctl->upd;
        auto loc = [&](int pos) { return pos >= 0 ? (s.sW[pos] & PACK_MASK) >> 1 : 0; };
        up[0] = 1;
        up[1] = c;
        up[2] = xa; up[3] = ya; up[4] = xb; up[5] = yb;
        up[6] = (a == b && ia == jb) ? 1 : 0;
        up[7] = s.sWoff[a] + ia + (b < a ? 1 : 0);
        up[8] = s.sWoff[b] + jb + (a <= b ? 1 : 0);
        up[9] = N;
        up[10] = Dx(t, s, loc(xa), c);
        up[11] = Dx(t, s, c, loc(ya));
        up[12] = Dx(t, s, loc(xb), c);
        up[13] = Dx(t, s, c, loc(yb));
        up[14] = Dx(t, s, c, c);
        up[15] = s.sp[c];
        ctl->incr = shortcut ? 0 : 1;
        ctl->sum_load = 0;                     // the route scans of the next step add it back up
        ctl->walks_done = 0;
    }
    __syncthreads();                           // every read of t.rem is done
    if (k0 + 1 < nrem) t.rem[k0] = remv;
    // more customers than threads (a route removal): the rest in chunks, the
    // loads of a chunk ahead of its stores
    for (int kb = blockDim.x; kb + 1 < nrem; kb += blockDim.x) {
        const int k = kb + threadIdx.x;
        const int v = k + 1 < nrem ? t.rem[k + (k >= pick ? 1 : 0)] : 0;
        __syncthreads();
        if (k + 1 < nrem) t.rem[k] = v;
    }
    if (threadIdx.x == 0) {
        ctl->nrem = nrem - 1;
        ctl->wsel ^= 1;
        ctl->n_short = 0;
    }
    __syncthreads();
}

// roulette wheel over enabled operators (fp64, explicit rounding)
__device__ int roulette(const double* w, const int* en, int k, double u) {
    double sum = 0.0;
    for (int i = 0; i < k; ++i)
        if (en[i]) sum = __dadd_rn(sum, w[i]);
    const double target = __dmul_rn(u, sum);
    double acc = 0.0;
    int last = -1;
    for (int i = 0; i < k; ++i) {
        if (!en[i]) continue;
        acc = __dadd_rn(acc, w[i]);
        last = i;
        if (target < acc) return i;
    }
    return last;
}

// Operator choice and removal size for iteration it (Algorithm 1, roulette
// wheels over the enabled operators); thread 0 of rank 0, right after the
// weight update of the previous iteration.
enum { D_RANDOM = 0, D_WORST = 1, D_SHAW = 2, D_CLUSTER = 3, D_ROUTE = 4, D_CRITICAL = 5, ND_OPS = 6 };

__device__ __noinline__ void pick_operators(const AlnsTeam& t, int it) {
    AlnsCtl* ctl = t.ctl;
    const unsigned long long base = static_cast<unsigned long long>(it) << 16;
    int en_d[ND_OPS];
    for (int i = 0; i < ND_OPS; ++i) en_d[i] = (t.destroy_mask >> i) & 1;
    const int en_r[4] = {(t.repair_mask & 1) != 0, (t.repair_mask & 2) != 0, (t.repair_mask & 4) != 0,
                         (t.repair_mask & 8) != 0};
    ctl->di = roulette(ctl->wd, en_d, ND_OPS, draw_unit(draw(t.key, base + 0)));
    ctl->rj = roulette(ctl->wr, en_r, 4, draw_unit(draw(t.key, base + 1)));
    ctl->ad[ctl->di] += 1;
    ctl->ar[ctl->rj] += 1;
    ctl->q = t.q_min + draw_below(draw(t.key, base + 2), t.q_max - t.q_min + 1);
}

// Ascending block-wide bitonic sort of P (a power of two) keys in shared memory.
__device__ void block_sort(unsigned long long* a, int P) {
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < P / 2; i += blockDim.x) {
                const int lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
                const bool asc = (lo & size) == 0;
                const unsigned long long x = a[lo], y = a[hi];
                if ((x > y) == asc) { a[lo] = y; a[hi] = x; }
            }
            __syncthreads();
        }
    }
}

// The structured destroy operators (Section 4.2.2), rank 0's block: marks
// s.flags[c] and leaves the count in ctl->q.  Rankings sort (key << 12 | c),
// so ties go to the smaller customer id.  Draws: the operator's pick at
// counter base + 4, sequential draws k at base + 16 + k.
__device__ __noinline__ void select_structured(const AlnsTeam& t, const Smem& s) {
    AlnsCtl* ctl = t.ctl;
    const int n = t.n, m = t.m, di = ctl->di, q = ctl->q, qmin = t.q_min;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned long long base = static_cast<unsigned long long>(ctl->iter) << 16;
    int P = 1;
    while (P < n) P <<= 1;
    const int rw = ((n + 1) + 3) & ~3;
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(s.rdy);      // [P]
    int* vd = s.rdy + 2 * P;                   // [n+1] vehicle of the dropoff
    int* vp = vd + rw;                         // [n+1] vehicle of the pickup
    int* tdr = vp + rw;                        // [n+1] dropoff time
    int* tpk = tdr + rw;                       // [n+1] pickup completion
    int* lst = tpk + rw;                       // [n+1] customer list
    int* sh = s.misc + 32;                     // scalars
    // facts of the current solution
    stage_ops(t, s, t.cur_ops, t.cur_off);
    const bool timed = di == D_SHAW || di == D_CRITICAL;
    if (timed && warp == 0) {
        int z;
        unsigned st;
        walk_depot(t, s, s.rdy, true, &z, &st);
    }
    __syncthreads();
    const int N = s.sWoff[m];
    for (int k = tid; k < N; k += blockDim.x) {
        int lo = 0, hi = m;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s.sWoff[mid] <= k) lo = mid; else hi = mid;
        }
        const int o = s.sW[k] & PACK_MASK, c = o >> 1;
        if (o & 1) { vp[c] = lo; if (timed) tpk[c] = t.H[k]; }
        else { vd[c] = lo; if (timed) tdr[c] = t.H[k]; }
    }
    __syncthreads();
    auto count_flags = [&]() {
        // every thread gets the number of marked customers
        __syncthreads();
        if (warp == 0) {
            int w = 0;
            for (int c0 = 1; c0 <= n; c0 += 32) w += __popc(__ballot_sync(FULL_MASK, c0 + lane <= n && s.flags[c0 + lane]));
            if (lane == 0) sh[1] = w;
        }
        __syncthreads();
        return sh[1];
    };
    auto take_sorted = [&](int need) {
        // mark the first `need` customers of the sorted keys (unmarked ones only carry keys)
        for (int i = tid; i < P && i < need; i += blockDim.x)
            if (keys[i] != KEY_NONE) s.flags[static_cast<int>(keys[i] & 0xFFF)] = 1;
    };
    if (di == D_WORST) {
        // removal gains from the team phase, largest first; q roulette draws
        // over the remaining ranked list with weight r^-6 on the r-th
        double* pw = reinterpret_cast<double*>(keys + P);                         // [n+1] prefix weights
        for (int i = tid; i < P; i += blockDim.x)
            keys[i] = i < n ? ((static_cast<unsigned long long>((1ll << 30) - t.gains[i + 1]) << 12) |
                               static_cast<unsigned long long>(i + 1))
                            : KEY_NONE;
        block_sort(keys, P);
        if (tid == 0) {
            double acc = 0.0;
            for (int r = 1; r <= n; ++r) {
                const double x = static_cast<double>(r), x2 = __dmul_rn(x, x);
                acc = __dadd_rn(acc, __ddiv_rn(1.0, __dmul_rn(__dmul_rn(x2, x2), x2)));
                pw[r] = acc;
            }
            for (int k = 0; k < q; ++k) {
                const int R = n - k;
                const double target = __dmul_rn(draw_unit(draw(t.key, base + 16 + static_cast<unsigned long long>(k))), pw[R]);
                int r = 1;
                while (r < R && !(pw[r] > target)) ++r;
                int seen = 0;
                for (int i = 0; i < n; ++i) {
                    const int c = static_cast<int>(keys[i] & 0xFFF);
                    if (s.flags[c]) continue;
                    if (++seen == r) { s.flags[c] = 1; break; }
                }
            }
        }
    } else if (di == D_SHAW || di == D_CLUSTER) {
        // a random seed and the q-1 customers nearest to it (Shaw: by the
        // relatedness measure, doubled to stay integral)
        if (tid == 0) sh[0] = 1 + draw_below(draw(t.key, base + 4), n);
        __syncthreads();
        const int sd = sh[0];
        for (int i = tid; i < P; i += blockDim.x) {
            const int c = i + 1;
            unsigned long long kk = KEY_NONE;
            if (c <= n && c != sd) {
                long long k2 = Dx(t, s, sd, c);
                if (di == D_SHAW) {
                    long long dt = static_cast<long long>(tdr[sd]) - tdr[c];
                    dt = dt < 0 ? -dt : dt;
                    k2 = 18 * k2 + 6 * dt + 5 * (vd[sd] != vd[c]) + 5 * (vp[sd] != vp[c]);
                }
                kk = (static_cast<unsigned long long>(k2) << 12) | static_cast<unsigned long long>(c);
            }
            keys[i] = kk;
        }
        block_sort(keys, P);
        if (tid == 0) s.flags[sd] = 1;
        take_sorted(q - 1);
    } else {
        // a random non-empty route, or the bottleneck route's customers
        if (tid == 0) {
            if (di == D_ROUTE) {
                int K = 0;
                for (int v = 0; v < m; ++v) K += s.sWoff[v + 1] > s.sWoff[v] ? 1 : 0;
                int kk = draw_below(draw(t.key, base + 4), K);
                int vsel = 0;
                for (int v = 0; v < m; ++v)
                    if (s.sWoff[v + 1] > s.sWoff[v] && kk-- == 0) { vsel = v; break; }
                sh[0] = vsel;
            } else {
                // latest return, the lower index on ties; q of its customers by
                // partial Fisher-Yates in customer order (all if fewer)
                long long best = -1;
                int vb = 0;
                for (int v = 0; v < m; ++v) {
                    long long rv = 0;
                    if (s.sWoff[v + 1] > s.sWoff[v]) {
                        const int last = s.sWoff[v + 1] - 1;
                        rv = static_cast<long long>(t.H[last]) + Dx(t, s, (s.sW[last] & PACK_MASK) >> 1, 0);
                    }
                    if (rv > best) { best = rv; vb = v; }
                }
                int nl = 0;
                for (int c = 1; c <= n; ++c)
                    if (vd[c] == vb || vp[c] == vb) lst[nl++] = c;
                const int take = q < nl ? q : nl;
                for (int k = 0; k < take; ++k) {
                    const int jj = k + draw_below(draw(t.key, base + 16 + static_cast<unsigned long long>(k)), nl - k);
                    const int tmp = lst[k];
                    lst[k] = lst[jj];
                    lst[jj] = tmp;
                    s.flags[lst[k]] = 1;
                }
                sh[0] = -1;
            }
        }
        __syncthreads();
        if (di == D_ROUTE) {
            const int vsel = sh[0];
            for (int k = s.sWoff[vsel] + tid; k < s.sWoff[vsel + 1]; k += blockDim.x)
                s.flags[(s.sW[k] & PACK_MASK) >> 1] = 1;
        }
        const int cnt = count_flags();
        if (cnt < qmin) {
            // top up: route removal by the least travel time from a removed
            // customer, critical path by the latest pickup completion
            if (di == D_ROUTE && warp == 0) {
                int w = 0;
                for (int c0 = 1; c0 <= n; c0 += 32) {
                    const int c = c0 + lane;
                    const bool r = c <= n && s.flags[c];
                    const unsigned bal = __ballot_sync(FULL_MASK, r);
                    if (r) lst[w + __popc(bal & ((1u << lane) - 1u))] = c;
                    w += __popc(bal);
                }
            }
            __syncthreads();
            for (int i = tid; i < P; i += blockDim.x) {
                const int c = i + 1;
                unsigned long long kk = KEY_NONE;
                if (c <= n && !s.flags[c]) {
                    long long k2;
                    if (di == D_ROUTE) {
                        k2 = 0x7fffffffll;
                        for (int j = 0; j < cnt; ++j) k2 = min(k2, static_cast<long long>(Dx(t, s, lst[j], c)));
                    } else {
                        k2 = (1ll << 30) - tpk[c];
                    }
                    kk = (static_cast<unsigned long long>(k2) << 12) | static_cast<unsigned long long>(c);
                }
                keys[i] = kk;
            }
            block_sort(keys, P);
            take_sorted(qmin - cnt);
        }
    }
    const int total = count_flags();
    if (tid == 0) ctl->q = total;
    __syncthreads();
}

// Rank 0: the destroy step (operator and q drawn at the end of the previous
// iteration), W = cur - removed.
// W[0] = the current solution without the customers flagged in s.flags:
// block-wide scan of the kept ops.  All threads of the block.
__device__ void build_W_from_cur(const AlnsTeam& t, const Smem& s) {
    const int m = t.m, two_n = 2 * t.n;
    const int per = (two_n + blockDim.x - 1) / blockDim.x;
    const int k0 = threadIdx.x * per, k1 = min(two_n, k0 + per);
    int cnt = 0;
    for (int k = k0; k < k1; ++k) cnt += s.flags[t.cur_ops[k] >> 1] ? 0 : 1;
    int* wsum = s.misc;                        // [ALNS_WARPS]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL_MASK, incl, o);
        if (lane >= o) incl += y;
    }
    __syncthreads();                           // wsum is free
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    int before = 0, kept_total = 0;
    for (int w = 0; w < ALNS_WARPS; ++w) {
        before += w < warp ? wsum[w] : 0;
        kept_total += wsum[w];
    }
    const int base_pos = before + incl - cnt;
    int pos = base_pos;
    int* Wn = t.W_ops[0];
    for (int k = k0; k < k1; ++k) {
        const int o = t.cur_ops[k];
        if (!s.flags[o >> 1]) Wn[pos++] = o;
    }
    // route offsets: the kept-op count before each route start, taken from the
    // scan by the thread whose range holds that start
    for (int v = 0; v <= m; ++v) {
        const int ov = t.cur_off[v];
        if (ov >= k0 && ov < k1) {
            int kept = base_pos;
            for (int k = k0; k < ov; ++k) kept += s.flags[t.cur_ops[k] >> 1] ? 0 : 1;
            t.W_off[0][v] = kept;
        } else if (ov == two_n && threadIdx.x == 0) {
            t.W_off[0][v] = kept_total;
        }
    }
    __syncthreads();
}

__device__ __noinline__ void phase_begin(const AlnsTeam& t, const Smem& s) {
    AlnsCtl* ctl = t.ctl;
    const int n = t.n;
    int* perm = s.rdy;                         // [n], shared memory
    for (int k = threadIdx.x; k < n; k += blockDim.x) perm[k] = k + 1;
    for (int c = threadIdx.x; c <= n; c += blockDim.x) s.flags[c] = 0;
    __syncthreads();
    if (threadIdx.x == 0 && ctl->di == D_RANDOM) {
        const int it = ctl->iter;
        const unsigned long long base = static_cast<unsigned long long>(it) << 16;
        const int q = ctl->q;
        for (int k = 0; k < q; ++k) {
            const int jj = k + draw_below(draw(t.key, base + 16 + static_cast<unsigned long long>(k)), n - k);
            const int tmp = perm[k];
            perm[k] = perm[jj];
            perm[jj] = tmp;
            s.flags[perm[k]] = 1;
        }
    }
    __syncthreads();
    if (ctl->di != D_RANDOM) select_structured(t, s);
    if (threadIdx.x == 0) {
        ctl->repair_fail = 0;
        ctl->n_short = 0;
        ctl->work_counter = 0;
        ctl->wsel = 0;
        ctl->incr = 0;                         // W lost customers: the next step walks it in full
        ctl->sum_load = 0;
        ctl->walks_done = 0;
    }
    __syncthreads();
    // removed customers in ascending id order (ballot compaction by warp 0)
    if ((threadIdx.x >> 5) == 0) {
        const int lane = threadIdx.x & 31;
        int w = 0;
        for (int c0 = 1; c0 <= n; c0 += 32) {
            const int c = c0 + lane;
            const bool r = c <= n && s.flags[c];
            const unsigned bal = __ballot_sync(FULL_MASK, r);
            if (r) t.rem[w + __popc(bal & ((1u << lane) - 1u))] = c;
            w += __popc(bal);
        }
        if (lane == 0) ctl->nrem = w;
    }
    build_W_from_cur(t, s);
}

// Rank 0: evaluate the repaired W and apply Algorithm 1's acceptance, cooling,
// reheat and weight update.  With first = true only records the start.
__device__ __noinline__ void phase_end(const AlnsTeam& t, const Smem& s, bool first) {
    AlnsCtl* ctl = t.ctl;
    const int n = t.n, m = t.m;
    stage_W(t, s);
    int* rdy = s.rdy;
    if ((threadIdx.x >> 5) == 0) {
        int z;
        unsigned st;
        walk_depot(t, s, rdy, false, &z, &st);
        if ((threadIdx.x & 31) == 0) {
            if (ctl->repair_fail) { z = 0x7fffffff; st = VRPRPD_MALFORMED; }
            ctl->z_work = z;
            ctl->st_work = st;
        }
    }
    __syncthreads();
    int* decision = s.misc;
    if (threadIdx.x == 0) {
        const int zn = ctl->z_work;
        const unsigned st = ctl->st_work;
        int accept = 0, newbest = 0;
        if (first) {
            accept = 1;
            newbest = 1;
            ctl->z_cur = zn;
            ctl->z_best = zn;
            ctl->z_init = zn;
            ctl->T = __dmul_rn(t.T0, static_cast<double>(zn));
            ctl->T_init = ctl->T;
            if (st != 0u) atomicExch(&ctl->err, DEV_BAD_STATE);
        } else {
            const int it = ctl->iter;
            const unsigned long long base = static_cast<unsigned long long>(it) << 16;
            const int di = ctl->di, rj = ctl->rj;
            if (st != 0u) {
                ctl->rejected += 1;
            } else if (zn < ctl->z_cur) {
                accept = 1;
                ctl->z_cur = zn;
                ctl->sd[di] += t.sigma2;
                ctl->sr[rj] += t.sigma2;
                ctl->improved += 1;
                ctl->accepted += 1;
                if (zn < ctl->z_best) {
                    newbest = 1;
                    ctl->z_best = zn;
                    ctl->sd[di] += t.sigma1 - t.sigma2;
                    ctl->sr[rj] += t.sigma1 - t.sigma2;
                    ctl->stagnation = 0;
                    ctl->new_best += 1;
                }
            } else {
                const double x = -__ddiv_rn(static_cast<double>(static_cast<long long>(zn) - ctl->z_cur), ctl->T);
                const double u = draw_unit(draw(t.key, base + 3));
                if (u < exp_sa(x)) {
                    accept = 1;
                    ctl->z_cur = zn;
                    ctl->sd[di] += t.sigma3;
                    ctl->sr[rj] += t.sigma3;
                    ctl->accepted += 1;
                }
            }
            ctl->T = __dmul_rn(t.alpha, ctl->T);
            ctl->stagnation += 1;
            if (ctl->stagnation >= t.stagnation_limit && ctl->T < __dmul_rn(0.01, ctl->T_init)) {
                ctl->T = __dmul_rn(__dmul_rn(t.reheat, t.T0), static_cast<double>(ctl->z_best));
                ctl->stagnation = 0;
                ctl->reheats += 1;
            }
            if (it % t.tau == 0) {
                for (int i = 0; i < ND_OPS; ++i) {
                    const double ratio = ctl->ad[i] ? __ddiv_rn(static_cast<double>(ctl->sd[i]), static_cast<double>(ctl->ad[i])) : 0.0;
                    const double w = __dadd_rn(__dmul_rn(__dsub_rn(1.0, t.r), ctl->wd[i]), __dmul_rn(t.r, ratio));
                    ctl->wd[i] = w < t.w_min ? t.w_min : w;
                    ctl->sd[i] = 0;
                    ctl->ad[i] = 0;
                }
                for (int i = 0; i < 4; ++i) {
                    const double ratio = ctl->ar[i] ? __ddiv_rn(static_cast<double>(ctl->sr[i]), static_cast<double>(ctl->ar[i])) : 0.0;
                    const double w = __dadd_rn(__dmul_rn(__dsub_rn(1.0, t.r), ctl->wr[i]), __dmul_rn(t.r, ratio));
                    ctl->wr[i] = w < t.w_min ? t.w_min : w;
                    ctl->sr[i] = 0;
                    ctl->ar[i] = 0;
                }
            }
            if (t.trace) t.trace[it - 1] = ctl->z_cur;
        }
        decision[0] = accept;
        decision[1] = newbest;
        const int next = first ? 1 : ctl->iter + 1;
        if (next <= t.iterations) pick_operators(t, next);
    }
    __syncthreads();
    const int accept = decision[0], newbest = decision[1];
    const int* W = t.W_ops[ctl->wsel];
    const int* Wo = t.W_off[ctl->wsel];
    if (accept && !first) {
        for (int k = threadIdx.x; k < 2 * n; k += blockDim.x) t.cur_ops[k] = W[k];
        for (int v = threadIdx.x; v <= m; v += blockDim.x) t.cur_off[v] = Wo[v];
    }
    if (newbest) {
        for (int k = threadIdx.x; k < 2 * n; k += blockDim.x) t.best_ops[k] = W[k];
        for (int v = threadIdx.x; v <= m; v += blockDim.x) t.best_off[v] = Wo[v];
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// multi-instance checkpoints (Section 4.2.1): all teams of the launch meet
// ---------------------------------------------------------------------------
// Barrier over every CTA of the launch; bounded (about 2 s), sets ctl->err.
__device__ bool grid_barrier(const AlnsTeam& t, unsigned& ggen) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = &t.gbar[1];
        const unsigned total = gridDim.x;
        __threadfence();
        const unsigned arrived = atomicAdd(&t.gbar[0], 1u) + 1u;
        if (arrived == total) {
            t.gbar[0] = 0u;
            __threadfence();
            atomicExch(&t.gbar[1], ggen + 1u);
        } else {
            const uint64_t t0 = global_ns();
            while (*vgen == ggen) {
                if (global_ns() - t0 > t.ctl->wait_ns) {
                    atomicExch(&t.ctl->err, DEV_TIMEOUT_BARRIER);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    ggen += 1u;
    __syncthreads();
    return *reinterpret_cast<volatile int*>(&t.ctl->err) == 0;
}

// Rank 0 of each team, between two grid barriers: when the best of all teams
// (lowest index among equal bests) beats this team's best, it becomes this
// team's current and best solution.  Nothing writes a best solution between
// the two barriers, so every team reads the same ones.
__device__ __noinline__ void replica_import(const AlnsTeam& t, const Smem& s) {
    AlnsCtl* ctl = t.ctl;
    int* sh = s.misc;
    if (threadIdx.x == 0) {
        int g = 0, zg = *reinterpret_cast<volatile const int*>(&t.sib[0].ctl->z_best);
        for (int r = 1; r < t.nreplicas; ++r) {
            const int zr = *reinterpret_cast<volatile const int*>(&t.sib[r].ctl->z_best);
            if (zr < zg) { zg = zr; g = r; }
        }
        sh[0] = ctl->z_best > zg ? g : -1;
        sh[1] = zg;
    }
    __syncthreads();
    const int g = sh[0];
    if (g >= 0) {
        const int* bo = t.sib[g].best_ops;
        const int* bf = t.sib[g].best_off;
        for (int k = threadIdx.x; k < 2 * t.n; k += blockDim.x) {
            const int o = __ldcg(bo + k);
            t.cur_ops[k] = o;
            t.best_ops[k] = o;
        }
        for (int v = threadIdx.x; v <= t.m; v += blockDim.x) {
            const int o = __ldcg(bf + v);
            t.cur_off[v] = o;
            t.best_off[v] = o;
        }
        if (threadIdx.x == 0) {
            ctl->z_cur = sh[1];
            ctl->z_best = sh[1];
            ctl->stagnation = 0;
            ctl->imports += 1;
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// periodic local search (Section 4.2.6), on the current solution
// ---------------------------------------------------------------------------
// Each candidate customer c runs one team step (prep, gaps, shortcut walks,
// matrix) on W = cur - c with one or more masked slots for c: pickup
// repositioning has one slot whose only drop gap is c's own dropoff place;
// relocation has one slot per vehicle v other than the bottleneck, with both
// gaps on v.  Taking c out can leave one of its old routes over capacity; the
// matrix judges the receiving routes only, so a slot is kept only if every
// such route is one it writes to.  The pass's best move is
// the least (makespan, travel, customer, flat gap index) over all slots; it
// is applied if it lowers the makespan.
enum { LS_PICKUP = 1, LS_RELOCATE = 2 };

// Rank 0: the candidates of one pass, in ascending id.  Pickup repositioning:
// customers whose pickup is on a vehicle returning at 95% of the makespan or
// later (20 ret >= 19 z); relocation: customers with an op on the bottleneck
// vehicle (latest return, lower index on ties).
__device__ __noinline__ void ls_candidates(const AlnsTeam& t, const Smem& s, int mode) {
    AlnsCtl* ctl = t.ctl;
    const int n = t.n, m = t.m, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    stage_ops(t, s, t.cur_ops, t.cur_off);
    int* ret = s.misc + 32;                    // [32] return time per route
    for (int c = tid; c <= n; c += blockDim.x) s.flags[c] = 0;
    if (warp == 0) {
        int z;
        unsigned st;
        walk_depot(t, s, s.rdy, true, &z, &st);
        __syncwarp();
        int rv = 0;
        if (lane < m && s.sWoff[lane + 1] > s.sWoff[lane]) {
            const int last = s.sWoff[lane + 1] - 1;
            rv = t.H[last] + Dx(t, s, (s.sW[last] & PACK_MASK) >> 1, 0);
        }
        ret[lane] = rv;
        __syncwarp();
        if (lane == 0) {
            int b = 0;
            for (int v = 1; v < m; ++v)
                if (ret[v] > ret[b]) b = v;
            ctl->ls_bott = b;
            ctl->ls_have = 0;
        }
    }
    __syncthreads();
    const long long z = ctl->z_cur;
    const int bott = ctl->ls_bott, N = s.sWoff[m];
    for (int k = tid; k < N; k += blockDim.x) {
        int lo = 0, hi = m;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s.sWoff[mid] <= k) lo = mid; else hi = mid;
        }
        const int o = s.sW[k] & PACK_MASK;
        const bool cand = mode == LS_PICKUP ? ((o & 1) && 20ll * ret[lo] >= 19ll * z) : lo == bott;
        if (cand) s.flags[o >> 1] = 1;
    }
    __syncthreads();
    if (warp == 0) {
        int w = 0;
        for (int c0 = 1; c0 <= n; c0 += 32) {
            const int c = c0 + lane;
            const bool r = c <= n && s.flags[c];
            const unsigned bal = __ballot_sync(FULL_MASK, r);
            if (r) t.lscand[w + __popc(bal & ((1u << lane) - 1u))] = c;
            w += __popc(bal);
        }
        if (lane == 0) ctl->ls_ncand = w;
    }
    __syncthreads();
}

// Rank 0: W = cur - c for candidate k, the routes of W over capacity, its
// travel, and the slots with their masks.
__device__ __noinline__ void ls_setup(const AlnsTeam& t, const Smem& s, int mode, int k) {
    AlnsCtl* ctl = t.ctl;
    const int n = t.n, m = t.m, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int c = t.lscand[k];
    int* sh = s.misc + 32;                     // [0] drop position of c in cur, [1] bad-route mask
    unsigned long long* travel = reinterpret_cast<unsigned long long*>(s.misc + 40);
    for (int x = tid; x <= n; x += blockDim.x) s.flags[x] = x == c ? 1 : 0;
    for (int q = tid; q < 2 * n; q += blockDim.x)
        if (t.cur_ops[q] == 2 * c) sh[0] = q;
    if (tid == 0) {
        sh[1] = 0;
        *travel = 0ull;
        ctl->wsel = 0;
    }
    __syncthreads();
    const int pdrop = sh[0];
    build_W_from_cur(t, s);
    stage_W(t, s);
    __syncthreads();
    // per route: stock range of W (the minimal or the full start load) and travel
    for (int r = warp; r < m; r += ALNS_WARPS) {
        const int st = s.sWoff[r], en = s.sWoff[r + 1];
        int carry = 0, mn = 0, mx = 0;
        long long tr = 0;
        for (int base = st; base < en; base += 32) {
            const int q = base + lane;
            const bool in = q < en;
            const int w = in ? s.sW[q] : 0;
            int v = in ? (((w & PACK_MASK) & 1) ? 1 : -1) : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULL_MASK, v, o);
                if (lane >= o) v += y;
            }
            if (in) {
                mn = min(mn, carry + v);
                mx = max(mx, carry + v);
                tr += w >> PACK_SHIFT;
            }
            carry += __shfl_sync(FULL_MASK, v, 31);
        }
        for (int o = 16; o > 0; o >>= 1) {
            mn = min(mn, __shfl_xor_sync(FULL_MASK, mn, o));
            mx = max(mx, __shfl_xor_sync(FULL_MASK, mx, o));
            tr += __shfl_xor_sync(FULL_MASK, tr, o);
        }
        if (lane == 0) {
            int load = 0;
            if (!cap_ok(t, mn, mx, load)) atomicOr(&sh[1], 1 << r);
            if (en > st) tr += Dx(t, s, (s.sW[en - 1] & PACK_MASK) >> 1, 0);
            atomicAdd(travel, static_cast<unsigned long long>(tr));
        }
    }
    __syncthreads();
    if (tid == 0) {
        const unsigned bad = static_cast<unsigned>(sh[1]);
        const unsigned all = m == 32 ? 0xffffffffu : (1u << m) - 1u;
        int ns = 0;
        if (mode == LS_PICKUP) {
            int a = 0;
            for (int v = 0; v < m; ++v)
                if (t.cur_off[v] <= pdrop) a = v;
            const int ia = pdrop - t.cur_off[a];
            const int g1 = s.sWoff[a] + a + ia;
            const unsigned rest = bad & ~(1u << a);
            if (__popc(rest) <= 1) {
                t.lsmask[0] = make_int4(static_cast<int>(1u << a), static_cast<int>(rest ? rest : all), g1, 0);
                t.rem[0] = c;
                ns = 1;
            }
            ctl->ls_rt = g1 / TR;
        } else {
            for (int v = 0; v < m; ++v) {
                if (v == ctl->ls_bott || (bad & ~(1u << v)) != 0u) continue;
                t.lsmask[ns] = make_int4(static_cast<int>(1u << v), static_cast<int>(1u << v), -1, 0);
                t.rem[ns] = c;
                ++ns;
            }
            ctl->ls_rt = -1;
        }
        ctl->nrem = ns;
        ctl->ls = mode;
        ctl->ls_travel = static_cast<long long>(*travel);
        ctl->repair_fail = 0;
        ctl->n_short = 0;
        ctl->work_counter = 0;
        ctl->incr = 0;
        ctl->sum_load = 0;
        ctl->walks_done = 0;
    }
    __syncthreads();
}

// Rank 0 after a candidate's matrix: its best entry over the slots against
// the pass's best move so far.
__device__ __noinline__ void ls_collect(const AlnsTeam& t, const Smem& s) {
    AlnsCtl* ctl = t.ctl;
    const int m = t.m, N = s.sWoff[m], G = N + m, ns = ctl->nrem, lane = threadIdx.x & 31;
    if ((threadIdx.x >> 5) == 0) {
        for (int ti = 0; ti < ns; ++ti) {
            unsigned long long bv = lane < m ? t.rkeys[ti * 32 + lane] : KEY_NONE;
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long other = __shfl_xor_sync(FULL_MASK, bv, o);
                bv = other < bv ? other : bv;
            }
            if (lane == 0 && bv != KEY_NONE) {
                const int row = static_cast<int>(bv & 0xFFF);
                const int col = static_cast<int>(t.keys[static_cast<long long>(ti) * G + row] & 0xFFF);
                const int dz = static_cast<int>(static_cast<unsigned>(bv >> 32) ^ 0x80000000u);
                const int dt = static_cast<int>((bv >> 12) & 0xFFFFFull) - (1 << 19);
                const int zn = ctl->z_work + dz;
                const long long tn = ctl->ls_travel + dt;
                const long long flat = static_cast<long long>(row) * G + col;
                const int c = t.rem[ti];
                bool better = !ctl->ls_have;
                if (!better) {
                    if (zn != ctl->ls_bz) better = zn < ctl->ls_bz;
                    else if (tn != ctl->ls_bt) better = tn < ctl->ls_bt;
                    else if (c != ctl->ls_c) better = c < ctl->ls_c;
                    else better = flat < ctl->ls_bflat;
                }
                if (better) {
                    ctl->ls_have = 1;
                    ctl->ls_c = c;
                    ctl->ls_bz = zn;
                    ctl->ls_bt = tn;
                    ctl->ls_bflat = flat;
                    ctl->ls_a = t.groute[row];
                    ctl->ls_ia = t.gpos[row];
                    ctl->ls_b = t.groute[col];
                    ctl->ls_jb = t.gpos[col];
                }
            }
        }
    }
    __syncthreads();
}

// Rank 0 at the end of a pass: apply the best move if it lowers the makespan.
__device__ __noinline__ void ls_apply(const AlnsTeam& t, const Smem& s) {
    AlnsCtl* ctl = t.ctl;
    const bool go = ctl->ls_have && ctl->ls_bz < ctl->z_cur;
    if (go) {
        const int c = ctl->ls_c;
        for (int x = threadIdx.x; x <= t.n; x += blockDim.x) s.flags[x] = x == c ? 1 : 0;
        if (threadIdx.x == 0) ctl->wsel = 0;
        __syncthreads();
        build_W_from_cur(t, s);
        stage_W(t, s);
        __syncthreads();
        insert_staged(t, s, c, ctl->ls_a, ctl->ls_ia, ctl->ls_b, ctl->ls_jb, t.cur_ops, t.cur_off);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ctl->ls_moved = go ? 1 : 0;
        ctl->ls = 0;
        if (go) {
            ctl->z_cur = ctl->ls_bz;
            ctl->ls_moves += 1;
        }
    }
    __syncthreads();
}

// Rank 0 after the local search of iteration it: the trace and the best solution.
__device__ __noinline__ void ls_finish(const AlnsTeam& t, const Smem& s, int it) {
    AlnsCtl* ctl = t.ctl;
    int* flag = s.misc;
    if (threadIdx.x == 0) {
        flag[0] = ctl->z_cur < ctl->z_best ? 1 : 0;
        if (flag[0]) {
            ctl->z_best = ctl->z_cur;
            ctl->stagnation = 0;
            ctl->ls_new_best += 1;
        }
        if (t.trace && it > 0) t.trace[it - 1] = ctl->z_cur;
    }
    __syncthreads();
    if (flag[0]) {
        for (int k = threadIdx.x; k < 2 * t.n; k += blockDim.x) t.best_ops[k] = t.cur_ops[k];
        for (int v = threadIdx.x; v <= t.m; v += blockDim.x) t.best_off[v] = t.cur_off[v];
    }
    __syncthreads();
}

// The local search of one iteration (it = 0: outside the iterations), every
// CTA of the team: up to three passes of each mode in lsm, pickup
// repositioning first.  False when a team barrier gave up.
__device__ __noinline__ bool ls_block(const AlnsTeam& t, const Smem& s, int rank, int team_blocks, unsigned& gen, int lsm, int it) {
    AlnsCtl* ctl = t.ctl;
    for (int mode = LS_PICKUP; mode <= LS_RELOCATE; ++mode) {
        if (!(lsm & mode)) continue;
        for (int pass = 0; pass < 3; ++pass) {
            if (rank == 0) ls_candidates(t, s, mode);
            if (!team_barrier(ctl, team_blocks, gen)) return false;
            const int ncand = *reinterpret_cast<volatile int*>(&ctl->ls_ncand);
            for (int k = 0; k < ncand; ++k) {
                if (rank == 0) ls_setup(t, s, mode, k);
                if (!team_barrier(ctl, team_blocks, gen)) return false;
                if (*reinterpret_cast<volatile int*>(&ctl->nrem) == 0) continue;
                phase_prep(t, s, rank, team_blocks, false);
                if (!team_barrier(ctl, team_blocks, gen)) return false;
                phase_gaps(t, s, rank, team_blocks);
                team_arrive(ctl, team_blocks, gen);
                gap_walks(t, s, rank, team_blocks);
                if (!team_wait(ctl, team_blocks, gen)) return false;
                phase_matrix(t, s);
                if (!team_barrier(ctl, team_blocks, gen)) return false;
                if (rank == 0) ls_collect(t, s);
            }
            if (rank == 0) ls_apply(t, s);
            if (!team_barrier(ctl, team_blocks, gen)) return false;
            if (!*reinterpret_cast<volatile int*>(&ctl->ls_moved)) break;
        }
    }
    if (rank == 0) ls_finish(t, s, it);
    return team_barrier(ctl, team_blocks, gen);
}

// The team barrier after the matrix phase, with the selection folded in: the
// CTA that arrives last (every tile and shortcut item of the step is then
// done and visible) selects and applies the insertion before it releases the
// others, so a greedy step crosses one barrier here instead of two.  Bounded
// like team_barrier; false when a wait gave up.
__device__ bool team_barrier_select(const AlnsTeam& t, const Smem& s, int team_blocks, unsigned& gen) {
    AlnsCtl* ctl = t.ctl;
    __shared__ int last;
    __syncthreads();
    if (team_blocks == 1) {
        phase_select(t, s);
        __syncthreads();
        return *reinterpret_cast<volatile int*>(&ctl->err) == 0;
    }
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned arrived = atomicAdd(&ctl->bar_count, 1u) + 1u;
        last = arrived == static_cast<unsigned>(team_blocks) ? 1 : 0;
        if (last) __threadfence();
    }
    __syncthreads();
    if (last) {
        phase_select(t, s);
        __syncthreads();
        if (threadIdx.x == 0) {
            ctl->bar_count = 0u;
            __threadfence();
            atomicExch(&ctl->bar_gen, gen + 1u);
        }
    } else if (threadIdx.x == 0) {
        volatile unsigned* vgen = &ctl->bar_gen;
        const uint64_t t0 = global_ns();
        while (*vgen == gen) {
            if (global_ns() - t0 > ctl->wait_ns) {
                atomicExch(&ctl->err, DEV_TIMEOUT_BARRIER);
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
    }
    gen += 1u;
    __syncthreads();
    return *reinterpret_cast<volatile int*>(&ctl->err) == 0;
}

__global__ void __launch_bounds__(ALNS_THREADS, 3) alns_kernel(AlnsTeam* teams, int team_blocks) {
    extern __shared__ __align__(16) int smem_alns[];
    __shared__ AlnsTeam team_s;
    const int team = blockIdx.x / team_blocks, rank = blockIdx.x - team * team_blocks;
    if (threadIdx.x == 0) team_s = teams[team];
    __syncthreads();
    const AlnsTeam& t = team_s;
    AlnsCtl* ctl = t.ctl;
    const Smem s = carve(smem_alns, t.n, t.m);   // coordinates follow the flags when staged
    for (int c = threadIdx.x; c <= t.n; c += blockDim.x) s.sp[c] = t.p[c];
    if (t.coords)
        for (int i = threadIdx.x; i < 2 * (t.n + 1); i += blockDim.x) s.xy[i] = t.coords[i];
    unsigned gen = 0, ggen = 0;
    __syncthreads();

    if (t.mode == 1) {
        // one-customer matrix dump on the partial solution already in W[0]
        if (!team_barrier(ctl, team_blocks, gen)) return;
        phase_prep(t, s, rank, team_blocks, false);
        if (!team_barrier(ctl, team_blocks, gen)) return;
        phase_gaps(t, s, rank, team_blocks);
        team_arrive(ctl, team_blocks, gen);
        gap_walks(t, s, rank, team_blocks);
        if (!team_wait(ctl, team_blocks, gen)) return;
        phase_matrix(t, s);
        team_barrier(ctl, team_blocks, gen);
        return;
    }
    if (t.mode == 3) {
        // repair steps on the partial solution already in W[0] (the search's
        // own step: prep, incrementally after a non-shortcut insertion, gaps,
        // shortcut walks, matrix, selection), then the matrix of the first
        // customer still to insert written out as in mode 1
        if (!team_barrier(ctl, team_blocks, gen)) return;
        for (int step = 0; step <= t.dump_steps; ++step) {
            if (*reinterpret_cast<volatile int*>(&ctl->repair_fail) || *reinterpret_cast<volatile int*>(&ctl->nrem) == 0)
                return;
            const bool incr = *reinterpret_cast<volatile int*>(&ctl->incr) != 0;
            if (rank == 0 && threadIdx.x == 0) {
                if (incr) ctl->steps_incr += 1; else ctl->steps_full += 1;
            }
            phase_prep(t, s, rank, team_blocks, incr);
            if (incr) {
                __syncthreads();
                if (threadIdx.x == 0) {
                    int* q = team_s.H; team_s.H = team_s.H2; team_s.H2 = q;
                    q = team_s.T; team_s.T = team_s.T2; team_s.T2 = q;
                    q = team_s.Ms; team_s.Ms = team_s.Ms2; team_s.Ms2 = q;
                }
                __syncthreads();
            }
            if (!team_barrier(ctl, team_blocks, gen)) return;
            phase_gaps(t, s, rank, team_blocks);
            team_arrive(ctl, team_blocks, gen);
            gap_walks(t, s, rank, team_blocks);
            if (!team_wait(ctl, team_blocks, gen)) return;
            if (step == t.dump_steps) {
                __syncthreads();
                if (threadIdx.x == 0) team_s.mode = 1;
                __syncthreads();
                phase_matrix(t, s);
                team_barrier(ctl, team_blocks, gen);
                return;
            }
            phase_matrix(t, s);
            if (!team_barrier_select(t, s, team_blocks, gen)) return;
        }
        return;
    }
    // start: W = cur, evaluate
    if (rank == 0) {
        for (int k = threadIdx.x; k < 2 * t.n; k += blockDim.x) t.W_ops[0][k] = t.cur_ops[k];
        for (int v = threadIdx.x; v <= t.m; v += blockDim.x) t.W_off[0][v] = t.cur_off[v];
        if (threadIdx.x == 0) ctl->wsel = 0;
        __syncthreads();
        phase_end(t, s, true);
    }
    if (!team_barrier(ctl, team_blocks, gen)) return;
    if (t.mode == 2) {
        // refinement of a start solution: local-search rounds until one moves nothing
        for (int round = 0; round < t.refine_rounds; ++round) {
            const int before = *reinterpret_cast<volatile int*>(&ctl->ls_moves);
            if (!ls_block(t, s, rank, team_blocks, gen, LS_PICKUP | LS_RELOCATE, 0)) return;
            if (*reinterpret_cast<volatile int*>(&ctl->ls_moves) == before) break;
        }
        return;
    }
    // wall time per phase, read by rank 0 at each barrier exit
    uint64_t tmark = global_ns();
    auto mark = [&](int ph) {
        if (rank == 0 && threadIdx.x == 0) {
            const uint64_t now = global_ns();
            ctl->phase_ns[ph] += now - tmark;
            tmark = now;
        }
    };
    for (int it = 1; it <= t.iterations; ++it) {
        if (*reinterpret_cast<volatile int*>(&ctl->di) == D_WORST) {
            // worst removal needs every customer's removal gain: a team phase
            phase_gains(t, s, rank, team_blocks);
            if (!team_barrier(ctl, team_blocks, gen)) return;
        }
        if (rank == 0) {
            if (threadIdx.x == 0) ctl->iter = it;
            __syncthreads();
            phase_begin(t, s);
        }
        if (!team_barrier(ctl, team_blocks, gen)) return;
        mark(0);
        while (true) {
            const int nrem = *reinterpret_cast<volatile int*>(&ctl->nrem);
            const int fail = *reinterpret_cast<volatile int*>(&ctl->repair_fail);
            if (nrem == 0 || fail) break;
            const bool incr = *reinterpret_cast<volatile int*>(&ctl->incr) != 0;
            if (rank == 0 && threadIdx.x == 0) {
                if (incr) ctl->steps_incr += 1; else ctl->steps_full += 1;
            }
            phase_prep(t, s, rank, team_blocks, incr);
            if (incr) {
                // every CTA swaps its own copy of the pointers: the update wrote the second buffers
                __syncthreads();
                if (threadIdx.x == 0) {
                    int* q = team_s.H; team_s.H = team_s.H2; team_s.H2 = q;
                    q = team_s.T; team_s.T = team_s.T2; team_s.T2 = q;
                    q = team_s.Ms; team_s.Ms = team_s.Ms2; team_s.Ms2 = q;
                }
                __syncthreads();
            }
            if (!team_barrier(ctl, team_blocks, gen)) return;
            mark(1);
            phase_gaps(t, s, rank, team_blocks);
            team_arrive(ctl, team_blocks, gen);
            gap_walks(t, s, rank, team_blocks);
            if (!team_wait(ctl, team_blocks, gen)) return;
            mark(2);
            phase_matrix(t, s);
            if (!team_barrier_select(t, s, team_blocks, gen)) return;   // select runs inside
            mark(3);
            mark(4);
        }
        if (rank == 0) phase_end(t, s, false);
        if (!team_barrier(ctl, team_blocks, gen)) return;
        mark(5);
        const int lsm = (t.ls_pickup > 0 && it % t.ls_pickup == 0 ? LS_PICKUP : 0) |
                        (t.ls_relocate > 0 && it % t.ls_relocate == 0 ? LS_RELOCATE : 0);
        if (lsm) {
            if (!ls_block(t, s, rank, team_blocks, gen, lsm, it)) return;
            mark(6);
        }
        if (t.nreplicas > 1 && t.sync_every > 0 && it % t.sync_every == 0) {
            if (!grid_barrier(t, ggen)) return;
            if (rank == 0) replica_import(t, s);
            if (!grid_barrier(t, ggen)) return;
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct DevBuf {
    char* base = nullptr;
    size_t used = 0, cap = 0;
    template <class T>
    T* take(size_t count) {
        size_t bytes = (count * sizeof(T) + 255) & ~static_cast<size_t>(255);
        T* p = reinterpret_cast<T*>(base + used);
        used += bytes;
        return p;
    }
};

static size_t team_bytes(int n, int m, int qmax, int iterations, bool dump) {
    const size_t N = 2ull * n, G = N + m;
    int levels = 1;
    while ((1ull << levels) <= N) ++levels;
    size_t w = 0;
    auto add = [&](size_t count, size_t sz) { w += (count * sz + 255) & ~static_cast<size_t>(255); };
    add(1, sizeof(AlnsCtl));
    add(N, 4); add(m + 1, 4); add(N, 4); add(m + 1, 4);
    add(N + 2, 4); add(m + 1, 4); add(N + 2, 4); add(m + 1, 4);
    add(std::max<size_t>(n + 1, qmax), 4); add(n + 1, 4);
    add(N, 4); add(N, 4); add(N * N, 4);
    add(N, 4); add(N, 4); add(N * N, 4);
    for (int i = 0; i < 5; ++i) add(N, 4);
    add(levels * N, 4); add(levels * N, 4);
    for (int i = 0; i < 12; ++i) add(G, 4);
    add(m, 4);
    add(G * 16, 4); add(G * 12, 4);
    add(static_cast<size_t>(qmax) * G, 16); add(static_cast<size_t>(qmax) * G, 16);
    add(static_cast<size_t>(qmax) * G, 8);
    add(static_cast<size_t>(qmax) * G, 8);
    add(static_cast<size_t>(qmax) * 32, 8);
    add(static_cast<size_t>(qmax) * 4, 8);
    add(static_cast<size_t>(qmax) * ((G + 31) / 32), 16);
    add(static_cast<size_t>(qmax) * G, 1);
    add(static_cast<size_t>(qmax) * G, 4);
    add(static_cast<size_t>(qmax) * G, 4);
    add(static_cast<size_t>(SC_CAP) * (4 * N + 8), 4);
    add(static_cast<size_t>(SC_CAP) * SC_CAP, 4);
    add(std::max(iterations, 1), 4);
    add(n + 1, 4);
    add(n + 1, 4); add(static_cast<size_t>(qmax), 16);
    if (dump) { add(G * G, 4); add(G * G, 4); }
    return w;
}

static void carve_team(AlnsTeam& t, DevBuf& B, int n, int m, int qmax, int iterations, bool dump) {
    const size_t N = 2ull * n, G = N + m;
    int levels = 1;
    while ((1ull << levels) <= N) ++levels;
    t.ctl = B.take<AlnsCtl>(1);
    t.cur_ops = B.take<int>(N); t.cur_off = B.take<int>(m + 1);
    t.best_ops = B.take<int>(N); t.best_off = B.take<int>(m + 1);
    t.W_ops[0] = B.take<int>(N + 2); t.W_off[0] = B.take<int>(m + 1);
    t.W_ops[1] = B.take<int>(N + 2); t.W_off[1] = B.take<int>(m + 1);
    t.rem = B.take<int>(std::max(n + 1, qmax)); t.perm = B.take<int>(n + 1);
    t.H = B.take<int>(N); t.T = B.take<int>(N); t.Ms = B.take<int>(N * N);
    t.H2 = B.take<int>(N); t.T2 = B.take<int>(N); t.Ms2 = B.take<int>(N * N);
    t.S_ = B.take<int>(N); t.PMINp = B.take<int>(N); t.PMAXp = B.take<int>(N);
    t.SMINs = B.take<int>(N); t.SMAXs = B.take<int>(N);
    t.spmin = B.take<int>(levels * N); t.spmax = B.take<int>(levels * N);
    t.log_levels = levels;
    t.gx = B.take<int>(G); t.gy = B.take<int>(G); t.gHx = B.take<int>(G); t.gTy = B.take<int>(G);
    t.gw = B.take<int>(G); t.gsb = B.take<int>(G); t.gpmin = B.take<int>(G); t.gpmax = B.take<int>(G);
    t.gsmin = B.take<int>(G); t.gsmax = B.take<int>(G); t.groute = B.take<int>(G); t.gpos = B.take<int>(G);
    t.rload = B.take<int>(m);
    t.growc = B.take<int>(G * 16); t.gcolc = B.take<int>(G * 12);
    t.vrow = B.take<int4>(static_cast<size_t>(qmax) * G); t.vcol = B.take<int4>(static_cast<size_t>(qmax) * G);
    t.vadj = B.take<int2>(static_cast<size_t>(qmax) * G);
    t.keys = B.take<unsigned long long>(static_cast<size_t>(qmax) * G);
    t.rkeys = B.take<unsigned long long>(static_cast<size_t>(qmax) * 32);
    t.gmin = B.take<unsigned long long>(static_cast<size_t>(qmax) * 4);
    t.band_stride = static_cast<int>((G + 31) / 32);
    t.bands = B.take<int4>(static_cast<size_t>(qmax) * t.band_stride);
    t.sc = B.take<unsigned char>(static_cast<size_t>(qmax) * G);
    t.slist = B.take<int>(static_cast<size_t>(qmax) * G);
    t.scix = B.take<int>(static_cast<size_t>(qmax) * G);
    t.scw_stride = static_cast<int>(4 * N + 8);
    t.scw = B.take<int>(static_cast<size_t>(SC_CAP) * (4 * N + 8));
    t.scpair = B.take<int>(static_cast<size_t>(SC_CAP) * SC_CAP);
    t.trace = B.take<int>(std::max(iterations, 1));
    t.gains = B.take<int>(n + 1);
    t.lscand = B.take<int>(n + 1);
    t.lsmask = B.take<int4>(static_cast<size_t>(qmax));
    t.dump_delta = dump ? B.take<int>(G * G) : nullptr;
    t.dump_travel = dump ? B.take<int>(G * G) : nullptr;
}

// Rows of the per-customer buffers: a route removal takes a whole route, so
// with that operator on, up to n customers wait for reinsertion at once; the
// relocation local search runs up to m - 1 slots for one customer.
int alns_row_cap(int n, int m, int qmax, const vrprpd_alns_params* P) {
    int cap = (P->destroy_mask & (1 << D_ROUTE)) ? n : qmax;
    if (P->ls_relocate_every > 0) cap = std::max(cap, m);
    return std::max(cap, 1);
}

// ALNS CTAs one SM holds for an instance of n customers and m vehicles (its
// shared memory with staged coordinates, the larger layout); 0 if none fits.
int alns_blocks_per_sm(int n, int m) {
    if (ensure_smem_limit(reinterpret_cast<const void*>(&alns_kernel))) return 0;
    int occ = 0;
    const size_t smem = alns_smem_words(n, m, true) * 4;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, alns_kernel, ALNS_THREADS, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return occ;
}

size_t alns_device_bytes(int n, int m, int qmax, const vrprpd_alns_params* P, int iterations) {
    const size_t R = static_cast<size_t>(std::max(1, P->replicas));
    return R * (team_bytes(n, m, alns_row_cap(n, m, qmax, P), iterations, false) + sizeof(AlnsTeam)) + 8192;
}

bool alns_supported(const vrprpd_instance* I, std::string* why) {
    if (I->m > 32) { *why = "ALNS needs m <= 32"; return false; }
    if (2 * I->n + I->m > 4096) { *why = "ALNS needs 2n + m <= 4096"; return false; }
    if (I->maxd >= (1 << 17)) { *why = "ALNS needs max d < 2^17"; return false; }
    // every schedule time of every insertion the matrix scores stays below
    // 2^27, so sums of three of them next to the exclusion sentinel fit int32
    const long long bound = (2ll * I->n + 1) * I->maxd + static_cast<long long>(I->n) * I->maxp;
    if (bound >= (1ll << 27)) { *why = "ALNS needs (2n+1)*max(d) + n*max(p) < 2^27"; return false; }
    return true;
}

static int choose_team_blocks(const vrprpd_instance* I, int requested, size_t smem, int nteams, int* out) {
    int occ = 0;
    { int rc_ = ensure_smem_limit(reinterpret_cast<const void*>(&alns_kernel)); if (rc_) return rc_; }
    VRP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, alns_kernel, ALNS_THREADS, smem));
    VRP_CHECK(occ > 0, VRPRPD_EINVAL, "ALNS block does not fit on an SM (n=%d)", I->n);
    // every CTA of every team is resident at once (a cooperative launch)
    const int maxb = occ * I->num_sms / nteams;
    VRP_CHECK(maxb >= 1, VRPRPD_EINVAL, "%d replicas exceed the %d resident ALNS blocks of this GPU", nteams,
              occ * I->num_sms);
    int tb = requested;
    if (tb <= 0) {
        // about one tile of the first step's matrix per CTA, at least one CTA
        const long long G = 2ll * I->n + I->m;
        const long long tiles = ((G + TR - 1) / TR) * ((G + TC - 1) / TC);
        tb = static_cast<int>(std::min<long long>(tiles, maxb));
        if (G < 64) tb = 1;
    }
    *out = std::max(1, std::min(tb, maxb));
    return VRPRPD_OK;
}

static int launch_alns(const vrprpd_instance* I, AlnsTeam* d_teams, int nteams, int team_blocks, size_t smem,
                       cudaStream_t stream) {
    void* args[] = {&d_teams, &team_blocks};
    const int grid = nteams * team_blocks;
    if (grid > 1) {
        VRP_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(&alns_kernel), dim3(grid),
                                             dim3(ALNS_THREADS), args, smem, stream));
    } else {
        alns_kernel<<<grid, ALNS_THREADS, smem, stream>>>(d_teams, team_blocks);
        VRP_CUDA(cudaGetLastError());
    }
    return VRPRPD_OK;
}

}  // namespace vrp

using namespace vrp;

extern "C" void vrprpd_alns_params_default(vrprpd_alns_params* P) {
    if (!P) return;
    P->T0 = 0.30;
    P->alpha = 0.9998;
    P->reheat = 0.50;
    P->r = 0.1;
    P->stagnation = 2000;
    P->tau = 100;
    P->sigma1 = 33;
    P->sigma2 = 9;
    P->sigma3 = 13;
    P->w_min = 0.1;
    P->q_min = 0;
    P->q_max = 0;
    P->iterations = 1000;
    P->repair_mask = 3;
    P->team_blocks = 0;
    P->destroy_mask = 1;
    P->ls_pickup_every = 200;
    P->ls_relocate_every = 500;
    P->replicas = 1;
    P->sync_every = 1000;
    P->init_mode = 1;
    P->init_refine_rounds = 10;
    P->wait_limit_ns = 2000000000ll;
}

// exact angular order around the depot: half plane, then cross product, then id
static bool angle_less(const std::vector<int32_t>& xy, int a, int b) {
    const long long ax = xy[2 * a] - xy[0], ay = xy[2 * a + 1] - xy[1];
    const long long bx = xy[2 * b] - xy[0], by = xy[2 * b + 1] - xy[1];
    const int ha = (ay < 0 || (ay == 0 && ax < 0)) ? 1 : 0, hb = (by < 0 || (by == 0 && bx < 0)) ? 1 : 0;
    if (ha != hb) return ha < hb;
    const long long cr = ax * by - ay * bx;
    if (cr != 0) return cr > 0;
    return a < b;
}

extern "C" int vrprpd_initial_solution(const vrprpd_instance* I, vrprpd_solution* out) {
    VRP_CHECK(I && out && out->ops && out->off, VRPRPD_EINVAL, "NULL argument");
    VRP_CHECK(I->R >= 1 && I->Q >= 1, VRPRPD_EINVAL, "initial solution needs R >= 1 and Q >= 1");
    const int n = I->n, m = I->m, N1 = n + 1;
    std::vector<int> order(n);
    for (int k = 0; k < n; ++k) order[k] = k + 1;
    if (I->has_coords)
        std::sort(order.begin(), order.end(), [&](int a, int b) { return angle_less(I->h_coords, a, b); });
    const int mact = std::min(m, I->R);
    const int b = std::max(1, std::min(I->Q, I->R / mact));
    long long W = 0;
    for (int k = 0; k < n; ++k) W += 2ll * I->h_d[order[k]] + I->h_p[order[k]];
    std::vector<int> sector(n);
    long long cum = 0;
    for (int k = 0; k < n; ++k) {
        const long long w = 2ll * I->h_d[order[k]] + I->h_p[order[k]];
        long long s = W > 0 ? ((2 * cum + w) * mact) / (2 * W) : (static_cast<long long>(k) * mact) / n;
        sector[k] = static_cast<int>(std::min<long long>(s, mact - 1));
        cum += w;
    }
    (void)N1;
    int w = 0;
    out->off[0] = 0;
    for (int v = 0; v < m; ++v) {
        std::vector<int> mine;
        for (int k = 0; k < n; ++k)
            if (sector[k] == v) mine.push_back(order[k]);
        for (size_t s = 0; s < mine.size(); s += b) {
            const size_t e = std::min(mine.size(), s + b);
            for (size_t q = s; q < e; ++q) out->ops[w++] = 2 * mine[q];
            for (size_t q = s; q < e; ++q) out->ops[w++] = 2 * mine[q] + 1;
        }
        out->off[v + 1] = w;
    }
    out->makespan = 0;
    out->status = 0;
    return VRPRPD_OK;
}

// Mode 3 (repair steps, then a matrix dump): the customers to insert, the
// repair operator, the steps, and where the partial solution goes afterwards.
struct RepairDump {
    int steps, op, count;
    const int32_t* removed;
    int32_t* out_ops;
    int32_t* out_off;
};

static int run_team(const vrprpd_instance* I, const vrprpd_solution* init, const vrprpd_alns_params* P,
                    uint64_t seed, int mode, int dump_c, const int32_t* dump_ops, const int32_t* dump_off,
                    vrprpd_solution* best, vrprpd_solution* current, vrprpd_alns_stats* stats, int32_t* trace,
                    int32_t* dump_delta, int32_t* dump_travel, cudaStream_t stream, int refine_rounds = 0,
                    const RepairDump* rd = nullptr) {
    std::string why;
    VRP_CHECK(alns_supported(I, &why), VRPRPD_EINVAL, "%s", why.c_str());
    const int n = I->n, m = I->m;
    int qmin = P->q_min, qmax = P->q_max;
    if (qmin <= 0 || qmax <= 0) {
        qmax = std::max(4, static_cast<int>(static_cast<long long>(n) * 5 / 100));
        qmin = std::max(4, qmax / 2);
    }
    qmax = std::min(qmax, n);
    qmin = std::min(qmin, qmax);
    VRP_CHECK(qmin >= 1 && qmax <= 1024, VRPRPD_EINVAL, "removal size must lie in [1, 1024] (q_min=%d q_max=%d)",
              qmin, qmax);
    const int iters = mode == 0 ? P->iterations : 0;
    VRP_CHECK(iters >= 0 && iters <= (1 << 24), VRPRPD_EINVAL, "iterations out of range");
    VRP_CHECK(P->tau >= 1, VRPRPD_EINVAL, "tau must be >= 1");
    VRP_CHECK(P->ls_pickup_every >= 0 && P->ls_relocate_every >= 0, VRPRPD_EINVAL,
              "local-search periods must be >= 0 (0 = off)");
    const bool dump = mode == 1 || mode == 3;
    const int R = mode != 0 ? 1 : std::max(1, P->replicas);
    VRP_CHECK(R <= 1024, VRPRPD_EINVAL, "replicas must lie in [0, 1024] (%d)", R);
    VRP_CHECK(P->sync_every >= 0, VRPRPD_EINVAL, "sync_every must be >= 0 (0 = never)");
    const int qcap = mode == 3 ? std::max(1, rd->count) : dump ? 1 : alns_row_cap(n, m, qmax, P);
    DevBuf B;
    const size_t per_team = team_bytes(n, m, qcap, iters, dump);
    B.cap = per_team * R + 4096;
    VRP_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&B.base), B.cap, stream));
    auto cleanup = [&]() { cudaFreeAsync(B.base, stream); };
    unsigned* gbar = B.take<unsigned>(4);
    AlnsTeam* d_team = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&d_team), sizeof(AlnsTeam) * R, stream);
    if (e != cudaSuccess) { cleanup(); set_error("alns setup: %s", cudaGetErrorString(e)); return VRPRPD_ECUDA; }
    AlnsTeam t{};
    t.n = n;
    t.m = m;
    t.R = I->R;
    t.Q = I->Q;
    t.load_full = (I->flags & VRPRPD_LOAD_FULL) != 0;
    t.d32 = I->d32;
    t.p = I->p;
    t.coords = coords_exact_small(I) ? I->coords : nullptr;
    t.T0 = P->T0;
    t.alpha = P->alpha;
    t.reheat = P->reheat;
    t.r = P->r;
    t.w_min = P->w_min;
    t.stagnation_limit = P->stagnation;
    t.tau = P->tau;
    t.sigma1 = P->sigma1;
    t.sigma2 = P->sigma2;
    t.sigma3 = P->sigma3;
    t.q_min = qmin;
    t.q_max = qmax;
    t.iterations = iters;
    t.repair_mask = P->repair_mask & 15;
    t.destroy_mask = P->destroy_mask & 63;
    t.ls_pickup = dump ? 0 : P->ls_pickup_every;
    t.ls_relocate = dump ? 0 : P->ls_relocate_every;
    auto fail_all = [&](int code) { cleanup(); cudaFreeAsync(d_team, stream); return code; };
    if (t.destroy_mask == 0) { set_error("destroy_mask enables no destroy operator"); return fail_all(VRPRPD_EINVAL); }
    if (t.repair_mask == 0) { set_error("repair_mask enables no repair operator"); return fail_all(VRPRPD_EINVAL); }
    t.mode = mode;
    t.refine_rounds = refine_rounds;
    t.dump_c = dump_c;
    t.dump_steps = mode == 3 ? rd->steps : 0;
    t.nreplicas = R;
    t.sync_every = P->sync_every;
    t.gbar = gbar;
    t.sib = d_team;
    // replica r draws from its own stream: the single-run stream for r = 0,
    // else a draw of it far past any iteration's counters
    const uint64_t key0 = stream_key(seed, RNG_STREAM_ALNS);
    std::vector<AlnsTeam> ts(R, t);
    for (int r = 0; r < R; ++r) {
        ts[r].replica = r;
        ts[r].key = r == 0 ? key0 : draw(key0, (0xFFFFFFFFull << 32) + static_cast<uint64_t>(r));
        carve_team(ts[r], B, n, m, qcap, iters, dump);
    }
    AlnsCtl ctl{};
    ctl.wait_ns = P->wait_limit_ns > 0 ? static_cast<unsigned long long>(P->wait_limit_ns) : 2000000000ull;
    for (int i = 0; i < 8; ++i) ctl.wd[i] = 1.0;
    ctl.wr[0] = ctl.wr[1] = ctl.wr[2] = ctl.wr[3] = 1.0;
    if (dump) {
        ctl.nrem = mode == 3 ? rd->count : 1;
        ctl.rj = mode == 3 ? rd->op : 0;
        ctl.wsel = 0;
    }
    e = cudaMemsetAsync(gbar, 0, 16, stream);
    for (int r = 0; r < R && e == cudaSuccess; ++r) e = cudaMemcpyAsync(ts[r].ctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice, stream);
    std::vector<int32_t> init_ops(2 * n), init_off(m + 1);
    if (!dump) {
        if (init) {
            std::memcpy(init_ops.data(), init->ops, 2 * n * 4);
            std::memcpy(init_off.data(), init->off, (m + 1) * 4);
        } else {
            vrprpd_solution s0{init_ops.data(), init_off.data(), 0, 0};
            const int rc = P->init_mode == 1
                               ? initial_solution_paper_tb(I, P->init_refine_rounds, &s0, stream, P->team_blocks)
                               : vrprpd_initial_solution(I, &s0);
            if (rc) return fail_all(rc);
        }
        for (int r = 0; r < R && e == cudaSuccess; ++r) {
            e = cudaMemcpyAsync(ts[r].cur_ops, init_ops.data(), 2 * n * 4, cudaMemcpyHostToDevice, stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(ts[r].cur_off, init_off.data(), (m + 1) * 4, cudaMemcpyHostToDevice, stream);
        }
    } else {
        const int Nops = dump_off[m];
        if (e == cudaSuccess) e = cudaMemcpyAsync(ts[0].W_ops[0], dump_ops, std::max(Nops, 1) * 4, cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ts[0].W_off[0], dump_off, (m + 1) * 4, cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess)
            e = mode == 3 ? cudaMemcpyAsync(ts[0].rem, rd->removed, rd->count * 4, cudaMemcpyHostToDevice, stream)
                          : cudaMemcpyAsync(ts[0].rem, &dump_c, 4, cudaMemcpyHostToDevice, stream);
        const size_t G = static_cast<size_t>(Nops) + (mode == 3 ? 2 * rd->steps : 0) + m;
        if (e == cudaSuccess) e = cudaMemsetAsync(ts[0].dump_delta, 0xff, G * G * 4, stream);
    }
    // recompute distances from staged coordinates only when that costs no resident CTAs
    size_t smem = alns_smem_words(n, m, false) * 4;
    if (t.coords) {
        const size_t smem_c = alns_smem_words(n, m, true) * 4;
        int occ0 = 0, occ1 = 0;
        ensure_smem_limit(reinterpret_cast<const void*>(&alns_kernel));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ0, alns_kernel, ALNS_THREADS, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ1, alns_kernel, ALNS_THREADS, smem_c);
        if (occ1 >= occ0 && smem_c <= I->smem_optin) smem = smem_c;
        else for (auto& x : ts) x.coords = nullptr;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_team, ts.data(), sizeof(AlnsTeam) * R, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) {
        set_error("alns setup: %s", cudaGetErrorString(e));
        return fail_all(VRPRPD_ECUDA);
    }
    if (smem > I->smem_optin) {
        set_error("ALNS shared memory %zu exceeds the limit", smem);
        return fail_all(VRPRPD_EINVAL);
    }
    int tb = 1;
    int rc = choose_team_blocks(I, P->team_blocks, smem, R, &tb);
    if (rc) return fail_all(rc);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, stream);
    rc = launch_alns(I, d_team, R, tb, smem, stream);
    cudaEventRecord(e1, stream);
    if (rc) return fail_all(rc);
    e = cudaStreamSynchronize(stream);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::vector<AlnsCtl> out(R);
    for (int r = 0; r < R && e == cudaSuccess; ++r) e = cudaMemcpyAsync(&out[r], ts[r].ctl, sizeof(AlnsCtl), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        set_error("alns run: %s", cudaGetErrorString(e));
        return fail_all(VRPRPD_ECUDA);
    }
    for (int r = 0; r < R; ++r) {
        if (out[r].err != 0) {
            set_error("alns device error %d (%s)", out[r].err,
                      out[r].err == DEV_TIMEOUT_BARRIER ? "team barrier timed out" : "inconsistent state");
            return fail_all(out[r].err == DEV_TIMEOUT_BARRIER ? VRPRPD_ETIMEOUT : VRPRPD_ECUDA);
        }
    }
    // the best of all replicas, the lowest index on ties; replica 0 reports
    // the current solution, the temperature and the weights
    int g = 0;
    for (int r = 1; r < R; ++r)
        if (out[r].z_best < out[g].z_best) g = r;
    if (mode == 3 && out[0].repair_fail) {
        set_error("a customer has no feasible insertion during the repair steps");
        return fail_all(VRPRPD_EINVAL);
    }
    if (dump) {
        const int Nout = dump_off[m] + (mode == 3 ? 2 * rd->steps : 0);
        const size_t G = static_cast<size_t>(Nout) + m;
        e = cudaMemcpyAsync(dump_delta, ts[0].dump_delta, G * G * 4, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess && mode == 3) {
            const int w = out[0].wsel;
            e = cudaMemcpyAsync(rd->out_ops, ts[0].W_ops[w], std::max(Nout, 1) * 4, cudaMemcpyDeviceToHost, stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(rd->out_off, ts[0].W_off[w], (m + 1) * 4, cudaMemcpyDeviceToHost, stream);
        }
        if (e == cudaSuccess && dump_travel) e = cudaMemcpyAsync(dump_travel, ts[0].dump_travel, G * G * 4, cudaMemcpyDeviceToHost, stream);
    } else {
        if (best) {
            e = cudaMemcpyAsync(best->ops, ts[g].best_ops, 2 * n * 4, cudaMemcpyDeviceToHost, stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(best->off, ts[g].best_off, (m + 1) * 4, cudaMemcpyDeviceToHost, stream);
            best->makespan = out[g].z_best;
            best->status = 0;
        }
        if (current && e == cudaSuccess) {
            e = cudaMemcpyAsync(current->ops, ts[0].cur_ops, 2 * n * 4, cudaMemcpyDeviceToHost, stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(current->off, ts[0].cur_off, (m + 1) * 4, cudaMemcpyDeviceToHost, stream);
            current->makespan = out[0].z_cur;
            current->status = 0;
        }
        for (int r = 0; r < R && trace && e == cudaSuccess && iters > 0; ++r)
            e = cudaMemcpyAsync(trace + static_cast<size_t>(r) * iters, ts[r].trace, iters * 4, cudaMemcpyDeviceToHost, stream);
    }
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->iterations = iters;
        for (int r = 0; r < R; ++r) {
            const AlnsCtl& o = out[r];
            stats->accepted += o.accepted;
            stats->improved += o.improved;
            stats->new_best += o.new_best;
            stats->reheats += o.reheats;
            stats->rejected_infeasible += o.rejected;
            stats->matrix_entries += static_cast<int64_t>(o.entries);
            stats->fallback_entries += static_cast<int64_t>(o.fallback_entries);
            stats->pruned_entries += static_cast<int64_t>(o.pruned);
            stats->tiles += static_cast<int64_t>(o.tiles);
            stats->tiles_pruned += static_cast<int64_t>(o.tiles_pruned);
            stats->incremental_steps += static_cast<int64_t>(o.steps_incr);
            stats->full_steps += static_cast<int64_t>(o.steps_full);
            stats->ls_moves += o.ls_moves;
            stats->ls_new_best += o.ls_new_best;
            stats->imports += o.imports;
        }
        stats->z_init = out[0].z_init;
        stats->z_best = out[g].z_best;
        stats->z_current = out[0].z_cur;
        stats->T_final = out[0].T;
        for (int i = 0; i < 8; ++i) stats->w_destroy[i] = i < ND_OPS ? out[0].wd[i] : 0.0;
        for (int i = 0; i < 4; ++i) stats->w_repair[i] = out[0].wr[i];
        stats->device_ms = ms;
        stats->team_blocks = tb;
        for (int i = 0; i < 6; ++i) stats->phase_ms[i] = static_cast<double>(out[0].phase_ns[i]) * 1e-6;
        stats->ls_ms = static_cast<double>(out[0].phase_ns[6]) * 1e-6;
        stats->replicas = R;
        stats->best_replica = g;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    cleanup();
    cudaFreeAsync(d_team, stream);
    if (e != cudaSuccess) {
        set_error("alns copy-out: %s", cudaGetErrorString(e));
        return VRPRPD_ECUDA;
    }
    return VRPRPD_OK;
}

extern "C" int vrprpd_initial_solution_paper(const vrprpd_instance* I, int32_t refine_rounds, vrprpd_solution* out,
                                             void* stream_) {
    return initial_solution_paper_tb(I, refine_rounds, out, static_cast<cudaStream_t>(stream_), 0);
}

namespace vrp {

int initial_solution_paper_tb(const vrprpd_instance* I, int32_t refine_rounds, vrprpd_solution* out,
                              cudaStream_t stream, int team_blocks) {
    VRP_CHECK(I && out && out->ops && out->off, VRPRPD_EINVAL, "NULL argument");
    VRP_CHECK(refine_rounds >= 0, VRPRPD_EINVAL, "refine_rounds must be >= 0");
    std::string why;
    VRP_CHECK(alns_supported(I, &why), VRPRPD_EINVAL, "%s", why.c_str());
    const int n = I->n, m = I->m;
    int32_t* dops = nullptr;
    VRP_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&dops), (2 * n + m + 1) * 4, stream));
    int32_t* doff = dops + 2 * n;
    int rc = construct_paper_device(I, dops, doff, stream);
    cudaError_t e = cudaSuccess;
    if (!rc) {
        e = cudaMemcpyAsync(out->ops, dops, 2 * n * 4, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out->off, doff, (m + 1) * 4, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    }
    cudaFreeAsync(dops, stream);
    if (rc) return rc;
    if (e != cudaSuccess) {
        set_error("initial solution: %s", cudaGetErrorString(e));
        return VRPRPD_ECUDA;
    }
    // evaluation and refinement in the ALNS kernel (refine-only mode)
    vrprpd_alns_params P;
    vrprpd_alns_params_default(&P);
    P.team_blocks = team_blocks;
    std::vector<int32_t> io(out->ops, out->ops + 2 * n), of(out->off, out->off + m + 1);
    vrprpd_solution start{io.data(), of.data(), 0, 0};
    return run_team(I, &start, &P, 0, 2, 0, nullptr, nullptr, nullptr, out, nullptr, nullptr, nullptr, nullptr,
                    stream, refine_rounds);
}

}  // namespace vrp

extern "C" int vrprpd_alns_run(const vrprpd_instance* I, const vrprpd_solution* init, const vrprpd_alns_params* P,
                               uint64_t seed, vrprpd_solution* best, vrprpd_solution* current,
                               vrprpd_alns_stats* stats, int32_t* z_trace, void* stream) {
    VRP_CHECK(I && P && best && best->ops && best->off, VRPRPD_EINVAL, "NULL argument");
    int rc = run_team(I, init, P, seed, 0, 0, nullptr, nullptr, best, current, stats, z_trace, nullptr, nullptr,
                      static_cast<cudaStream_t>(stream));
    return rc;
}

extern "C" int vrprpd_repair_then_matrix(const vrprpd_instance* I, const int32_t* ops, const int32_t* off,
                                         const int32_t* removed, int32_t count, int32_t repair_op, int32_t steps,
                                         int32_t team_blocks, int32_t* out_ops, int32_t* out_off, int32_t* delta,
                                         int32_t* travel, int64_t* incremental_steps, void* stream) {
    VRP_CHECK(I && ops && off && removed && out_ops && out_off && delta, VRPRPD_EINVAL, "NULL argument");
    const int m = I->m, n = I->n;
    VRP_CHECK(count >= 1 && count <= 1024, VRPRPD_EINVAL, "count must lie in [1, 1024]");
    VRP_CHECK(steps >= 0 && steps < count, VRPRPD_EINVAL, "steps must lie in [0, count)");
    VRP_CHECK(repair_op >= 0 && repair_op <= 3, VRPRPD_EINVAL, "repair_op must lie in [0, 3]");
    VRP_CHECK(off[0] == 0 && off[m] == 2 * (n - count), VRPRPD_EINVAL, "the partial solution must hold 2(n - count) ops");
    for (int v = 0; v < m; ++v) VRP_CHECK(off[v + 1] >= off[v], VRPRPD_EINVAL, "offsets decrease");
    std::vector<char> seen(2 * n + 2, 0);
    for (int k = 0; k < off[m]; ++k) {
        const int o = ops[k];
        VRP_CHECK(o >= 2 && o <= 2 * n + 1 && !seen[o], VRPRPD_EINVAL, "bad or repeated op %d", o);
        seen[o] = 1;
    }
    for (int k = 0; k < count; ++k) {
        const int c = removed[k];
        VRP_CHECK(c >= 1 && c <= n && (k == 0 || c > removed[k - 1]), VRPRPD_EINVAL,
                  "removed customers must be ascending ids in [1, n]");
        VRP_CHECK(!seen[2 * c] && !seen[2 * c + 1], VRPRPD_EINVAL, "customer %d is in the partial solution", c);
    }
    for (int q = 1; q <= n; ++q) VRP_CHECK(seen[2 * q] == seen[2 * q + 1], VRPRPD_EINVAL, "customer %d half present", q);
    vrprpd_alns_params P;
    vrprpd_alns_params_default(&P);
    P.team_blocks = team_blocks;
    RepairDump rd{steps, repair_op, count, removed, out_ops, out_off};
    vrprpd_alns_stats st;
    const int rc = run_team(I, nullptr, &P, 0, 3, 0, ops, off, nullptr, nullptr, &st, nullptr, delta, travel,
                            static_cast<cudaStream_t>(stream), 0, &rd);
    if (rc == VRPRPD_OK && incremental_steps) *incremental_steps = st.incremental_steps;
    return rc;
}

extern "C" int vrprpd_insertion_matrix(const vrprpd_instance* I, const int32_t* ops, const int32_t* off, int32_t c,
                                       int32_t* delta, int32_t* travel, void* stream) {
    VRP_CHECK(I && ops && off && delta, VRPRPD_EINVAL, "NULL argument");
    VRP_CHECK(c >= 1 && c <= I->n, VRPRPD_EINVAL, "customer %d out of range", c);
    const int m = I->m;
    VRP_CHECK(off[0] == 0 && off[m] >= 0 && off[m] <= 2 * I->n - 2, VRPRPD_EINVAL, "bad partial offsets");
    for (int v = 0; v < m; ++v) VRP_CHECK(off[v + 1] >= off[v], VRPRPD_EINVAL, "offsets decrease");
    std::vector<char> seen(2 * I->n + 2, 0);
    for (int k = 0; k < off[m]; ++k) {
        const int o = ops[k];
        VRP_CHECK(o >= 2 && o <= 2 * I->n + 1 && !seen[o], VRPRPD_EINVAL, "bad or repeated op %d", o);
        VRP_CHECK((o >> 1) != c, VRPRPD_EINVAL, "customer %d is already in the partial solution", c);
        seen[o] = 1;
    }
    for (int q = 1; q <= I->n; ++q) VRP_CHECK(seen[2 * q] == seen[2 * q + 1], VRPRPD_EINVAL, "customer %d half present", q);
    vrprpd_alns_params P;
    vrprpd_alns_params_default(&P);
    return run_team(I, nullptr, &P, 0, 1, c, ops, off, nullptr, nullptr, nullptr, nullptr, delta, travel,
                    static_cast<cudaStream_t>(stream));
}
