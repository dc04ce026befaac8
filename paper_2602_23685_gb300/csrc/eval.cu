// Batched candidate evaluation (the repair's timing evaluation of Section
// 4.2.3 and the decoder's schedule simulation of Section 4.4.2, done exactly
// on the semantics of Section 3.1, Eqs. 7-23).
//
// Batched form: a persistent launch; the block stages the instance (distances
// or coordinates, and p) in shared memory with TMA bulk copies, and every warp
// owns a tile of k = 32/m candidates (one lane per route).  Per tile:
//   1. offsets are checked and every customer's ready slot is set to
//      -(p_c + 1): negative means "not dropped yet", and the drop recovers p_c
//      from the value it reads anyway;
//   2. the ops are read with coalesced loads, four per lane in flight (int32
//      codes, or pairs of 16-bit codes in the 16-bit form), checked (code
//      range, duplicates by a shared bitmap) and kept as 16-bit codes:
//      half the footprint of the 32-bit stream, so 24 warps fit per SM where
//      a staged 32-bit copy left room for 16;
//   3. the route walk: each lane advances its route up to two ops per step,
//      computing each travel time from the previous stop -- a drop publishes
//      its pickup-ready time T_drop + p_c to shared memory, a pickup waits
//      until that time is published (cross-vehicle precedence, Eq. 9) and then
//      leaves at max(arrival, ready) (Eqs. 8, 10).  A group that makes no
//      progress in a step while unfinished is a precedence cycle.  Each lane
//      also tracks its route's stock prefix (Eqs. 13-18);
//   4. per-candidate reductions: makespan = max return time (Eqs. 21-22),
//      vehicle capacity, depot pool.
// Plain form: one thread per candidate, Kahn order over routes, scratch in
// global memory, distances from global memory.
#include <algorithm>
#include <cstring>

#include "device_common.cuh"
#include "internal.h"

namespace vrp {

struct EvalArgs {
    const int32_t* ops;
    const uint16_t* ops16;   // the 16-bit form (ops/off unused then)
    const uint16_t* off16;
    const int32_t* off;
    int32_t* z;
    uint32_t* st;
    const int32_t* d32;
    const uint16_t* d16;
    const int32_t* coords;
    const int32_t* p;
    int* err;
    long long num;
    int n, m, R, Q;
    int load_full;
    int k;            // candidates per warp tile
    int N;            // n + 1
    // shared-memory layout, in 32-bit words
    int shared_words; // per-block instance data (distances/coords + p)
    int dist_words;
    int a_words, ready_words, seen_words, start_words, off_words, valid_words, warp_words;
    int sw;           // seen words per candidate
    // streamed form: G warps per group, K candidates per group tile, and the
    // group region's layout in 32-bit words
    int G, K;
    int g_ready, g_off, g_flag, g_prog, g_red, group_words;
};

template <int DM>
__device__ __forceinline__ int dist(const EvalArgs& a, const int32_t* sh, int i, int j) {
    if constexpr (DM == VRPRPD_DIST_SMEM32) {
        return sh[i * a.N + j];
    } else if constexpr (DM == VRPRPD_DIST_SMEM16) {
        return reinterpret_cast<const uint16_t*>(sh)[i * a.N + j];
    } else if constexpr (DM == VRPRPD_DIST_GLOBAL16) {
        return __ldg(a.d16 + i * a.N + j);
    } else if constexpr (DM == VRPRPD_DIST_GLOBAL32) {
        return __ldg(a.d32 + i * a.N + j);
    } else {
        const int2 pi = reinterpret_cast<const int2*>(sh)[i];
        const int2 pj = reinterpret_cast<const int2*>(sh)[j];
        return euc2d_small(pi.x, pi.y, pj.x, pj.y);
    }
}

// One tile of k candidates of one instance, processed by one warp.
// W is the warp's shared-memory region (layout from a), sh/sp the block's
// staged distances or coordinates and p.
template <int DM, bool W16>
__device__ __forceinline__ bool eval_tile(const EvalArgs& a, const int32_t* sh, const int32_t* sp, int32_t* W,
                                          uint64_t* bar, unsigned& phase, long long t) {
    (void)bar;
    (void)phase;
    const int lane = threadIdx.x & 31;
    const int n = a.n, m = a.m, two_n = 2 * n, k = a.k;
    uint16_t* A = reinterpret_cast<uint16_t*>(W);            // op codes, 16 bits each
    int32_t* ready = W + a.a_words;
    uint32_t* seen = reinterpret_cast<uint32_t*>(ready + a.ready_words);
    int32_t* soff = reinterpret_cast<int32_t*>(seen + a.seen_words + a.start_words);
    int32_t* valid = soff + a.off_words;
    int32_t* red = valid + a.valid_words;      // 96 words
    const int grp = lane / m, v = lane - grp * m;
    const unsigned gmask = (grp < k) ? (m == 32 ? FULL_MASK : (((1u << m) - 1u) << (grp * m))) : 0u;
    const long long first = t * k;
    const int kt = static_cast<int>(min(static_cast<long long>(k), a.num - first));
    const int elems = kt * two_n;

    // ---- 1. offsets, flags, duplicate bitmap, unresolved ready times ----
    for (int i = lane; i < kt * (m + 1); i += 32)
        soff[i] = W16 ? static_cast<int32_t>(__ldg(a.off16 + first * (m + 1) + i)) : __ldg(a.off + first * (m + 1) + i);
    for (int i = lane; i < kt; i += 32) valid[i] = 1;
    for (int i = lane; i < kt * a.sw; i += 32) seen[i] = 0u;
    // unresolved ready time of c: -(p_c + 1) (negative); the drop recovers p_c from it
    for (int g = 0; g < kt; ++g)
        for (int c = lane; c <= n; c += 32) ready[g * (n + 1) + c] = -1 - sp[c];
    __syncwarp();
    // offsets: off[0] = 0, off[m] = 2n, non-decreasing
    for (int i = lane; i < kt * (m + 1); i += 32) {
        const int g = i / (m + 1), vv = i - g * (m + 1);
        const int val = soff[i];
        bool bad = val < 0 || val > two_n || (vv == 0 && val != 0) || (vv == m && val != two_n) ||
                   (vv < m && val > soff[i + 1]);
        if (bad) atomicAnd(&valid[g], 0);
    }

    // ---- 2. ops: coalesced loads, four in flight per lane; code range and
    // duplicates; kept as 16-bit codes (the walk computes the travel times) ----
    if constexpr (W16) {
        // code pairs as 32-bit words: 2n is even, so a pair never straddles
        // two candidates (n pairs each), and candidate i starts 4n i bytes in
        const uint32_t* src = reinterpret_cast<const uint32_t*>(a.ops16 + first * two_n);
        uint32_t* A2 = reinterpret_cast<uint32_t*>(A);
        const int pairs = elems >> 1;
        int gbase = 0;
        for (int base = 0; base < pairs; base += 128) {
            uint32_t raw[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = base + 32 * u + lane;
                raw[u] = e < pairs ? __ldg(src + e) : 0x00020002u;
            }
            if (k > 1)
                while ((gbase + 1) * n <= base) ++gbase;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = base + 32 * u + lane;
                if (e < pairs) {
                    int g = gbase;
                    if (k > 1)
                        while ((g + 1) * n <= e) ++g;
                    const int lo = static_cast<int>(raw[u] & 0xffffu), hi = static_cast<int>(raw[u] >> 16);
                    const bool okl = lo >= 2 && lo <= two_n + 1, okh = hi >= 2 && hi <= two_n + 1;
                    bool bad = !(okl && okh);
                    if (okl) {
                        const unsigned bit = 1u << (lo & 31);
                        bad |= (atomicOr(&seen[g * a.sw + (lo >> 5)], bit) & bit) != 0u;
                    }
                    if (okh) {
                        const unsigned bit = 1u << (hi & 31);
                        bad |= (atomicOr(&seen[g * a.sw + (hi >> 5)], bit) & bit) != 0u;
                    }
                    if (bad) atomicAnd(&valid[g], 0);
                    A2[e] = static_cast<uint32_t>(okl ? lo : 2) | (static_cast<uint32_t>(okh ? hi : 2) << 16);
                }
            }
        }
    } else {
        const int32_t* src = a.ops + first * two_n;
        int gbase = 0;
        for (int base = 0; base < elems; base += 128) {
            int raw[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = base + 32 * u + lane;
                raw[u] = e < elems ? __ldg(src + e) : 2;
            }
            if (k > 1)
                while ((gbase + 1) * two_n <= base) ++gbase;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = base + 32 * u + lane;
                if (e < elems) {
                    int g = gbase;
                    if (k > 1)
                        while ((g + 1) * two_n <= e) ++g;
                    const bool ok = raw[u] >= 2 && raw[u] <= two_n + 1;
                    bool bad = !ok;
                    if (ok) {
                        const unsigned bit = 1u << (raw[u] & 31);
                        bad = (atomicOr(&seen[g * a.sw + (raw[u] >> 5)], bit) & bit) != 0u;
                    }
                    if (bad) atomicAnd(&valid[g], 0);
                    A[e] = static_cast<uint16_t>(ok ? raw[u] : 2);
                }
            }
        }
    }
    __syncwarp();

    // ---- 3. route walk (branch-free; up to two ops per lane per step) ----
    // Each op's travel time is computed here from the previous stop.  Ready
    // times have a single writer (the dropping lane) and are read with
    // volatile loads: a pickup sees either "unresolved" (and retries next
    // step) or the final value.  The __syncwarp at the end of each step makes
    // every write of step t visible in step t+1, so a group with no progress
    // in a step can never progress again (a cycle).
    const bool mine = grp < kt && valid[grp] != 0;
    int pos = 0, end = 0, start = 0;
    if (mine) {
        start = pos = soff[grp * (m + 1) + v];
        end = soff[grp * (m + 1) + v + 1];
    }
    const uint16_t* wp = A + (grp < k ? grp : 0) * two_n;
    volatile int* rdy = ready + (grp < k ? grp : 0) * (n + 1);
    int dep = 0, s = 0, smin = 0, smax = 0, loc = 0;
    bool walking = mine && pos < end, cyc = false;
    while (__any_sync(FULL_MASK, walking)) {
        // first op
        const int o1 = walking ? wp[pos] : 0;
        const int c1 = o1 >> 1;
        const bool p1 = (o1 & 1) != 0;
        // Travel times from shared memory are computed branch-free on every
        // lane (an idle lane reads code 0, the depot; its result is unused);
        // with coordinates, c1's point is kept for the second op's leg.  Only
        // the L2 gathers are skipped on idle lanes.
        int2 pc1 = make_int2(0, 0);
        int t1;
        if constexpr (DM == VRPRPD_DIST_COORDS) {
            const int2 pl = reinterpret_cast<const int2*>(sh)[loc];
            pc1 = reinterpret_cast<const int2*>(sh)[c1];
            t1 = euc2d_small(pl.x, pl.y, pc1.x, pc1.y);
        } else if constexpr (DM == VRPRPD_DIST_SMEM32 || DM == VRPRPD_DIST_SMEM16) {
            t1 = dist<DM>(a, sh, loc, c1);
        } else {
            t1 = walking ? dist<DM>(a, sh, loc, c1) : 0;
        }
        const int r1 = rdy[c1];
        const bool go1 = walking && (!p1 || r1 >= 0);
        const int a1 = dep + t1;
        if (go1 && !p1) rdy[c1] = a1 - 1 - r1;
        dep = go1 ? max(a1, p1 ? r1 : 0) : dep;
        s += go1 ? (p1 ? 1 : -1) : 0;
        smin = min(smin, s);
        smax = max(smax, s);
        pos += go1 ? 1 : 0;
        loc = go1 ? c1 : loc;
        // second op, only behind a first one that went
        const bool try2 = go1 && pos < end;
        const int o2 = try2 ? wp[pos] : 0;
        const int c2 = o2 >> 1;
        const bool p2 = (o2 & 1) != 0;
        int t2;
        if constexpr (DM == VRPRPD_DIST_COORDS) {
            const int2 pc2 = reinterpret_cast<const int2*>(sh)[c2];
            t2 = euc2d_small(pc1.x, pc1.y, pc2.x, pc2.y);
        } else if constexpr (DM == VRPRPD_DIST_SMEM32 || DM == VRPRPD_DIST_SMEM16) {
            t2 = dist<DM>(a, sh, c1, c2);
        } else {
            t2 = try2 ? dist<DM>(a, sh, c1, c2) : 0;
        }
        const int r2 = rdy[c2];
        const bool go2 = try2 && (!p2 || r2 >= 0);
        const int a2 = dep + t2;
        if (go2 && !p2) rdy[c2] = a2 - 1 - r2;
        dep = go2 ? max(a2, p2 ? r2 : 0) : dep;
        s += go2 ? (p2 ? 1 : -1) : 0;
        smin = min(smin, s);
        smax = max(smax, s);
        pos += go2 ? 1 : 0;
        loc = go2 ? c2 : loc;
        const unsigned prog = __ballot_sync(FULL_MASK, go1);
        const bool more = pos < end;
        cyc = cyc || (walking && more && (prog & gmask) == 0u);
        walking = walking && more && !cyc;
        __syncwarp();
    }
    if (cyc)                                   // finish the stock prefix of a blocked route
        for (; pos < end; ++pos) {
            const int o = wp[pos];
            if (o & 1) { ++s; smax = max(smax, s); } else { --s; smin = min(smin, s); }
        }

    // ---- 4. per-candidate reduction ----
    int ret = 0, flags = 0, pool = 0;
    if (mine) {
        if (!cyc && end > start) ret = dep + dist<DM>(a, sh, loc, 0);
        if (a.load_full) {
            flags = (smin < -a.Q || smax > 0) ? VRPRPD_VEH_CAP : 0;
            pool = a.Q;
        } else {
            flags = (-smin + smax > a.Q) ? VRPRPD_VEH_CAP : 0;
            pool = -smin;
        }
        if (cyc) flags |= VRPRPD_CYCLE;
    }
    red[lane] = ret;
    red[32 + lane] = flags;
    red[64 + lane] = pool;
    __syncwarp();
    if (grp < kt && v == 0) {
        int z = 0, f = 0;
        long long pl = 0;
        for (int j = 0; j < m; ++j) {
            z = max(z, red[grp * m + j]);
            f |= red[32 + grp * m + j];
            pl += red[64 + grp * m + j];
        }
        if (pl > a.R) f |= VRPRPD_POOL;
        if (f & VRPRPD_CYCLE) z = 0x7fffffff;
        if (!valid[grp]) { z = 0x7fffffff; f = VRPRPD_MALFORMED; }
        a.z[first + grp] = z;
        a.st[first + grp] = static_cast<uint32_t>(f);
    }
    __syncwarp();
    return true;
}

template <int DM, bool W16>
__global__ void __launch_bounds__(1024) eval_tiles_kernel(EvalArgs a) {
    extern __shared__ __align__(16) int32_t smem[];
    __shared__ __align__(8) uint64_t block_bar;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;

    // ---- block-wide staging of the instance (TMA bulk copies) ----
    int32_t* sh = smem;                        // distances or coordinates
    int32_t* sp = smem + a.dist_words;         // p[0..n]
    if (threadIdx.x == 0) {
        mbar_init(&block_bar, 1);
        unsigned dist_bytes = 0;
        if constexpr (DM == VRPRPD_DIST_SMEM32) dist_bytes = ((a.N * a.N * 4) + 15) & ~15;
        if constexpr (DM == VRPRPD_DIST_SMEM16) dist_bytes = ((a.N * a.N * 2) + 15) & ~15;
        if constexpr (DM == VRPRPD_DIST_COORDS) dist_bytes = ((a.N * 8) + 15) & ~15;
        unsigned p_bytes = ((a.N * 4) + 15) & ~15;
        mbar_arrive_expect_tx(&block_bar, dist_bytes + p_bytes);
        if constexpr (DM == VRPRPD_DIST_SMEM32) tma_bulk_g2s(sh, a.d32, dist_bytes, &block_bar);
        if constexpr (DM == VRPRPD_DIST_SMEM16) tma_bulk_g2s(sh, a.d16, dist_bytes, &block_bar);
        if constexpr (DM == VRPRPD_DIST_COORDS) tma_bulk_g2s(sh, a.coords, dist_bytes, &block_bar);
        tma_bulk_g2s(sp, a.p, p_bytes, &block_bar);
    }
    __syncthreads();
    if (!mbar_wait_bounded(&block_bar, 0)) {
        if (threadIdx.x == 0) atomicExch(a.err, DEV_TIMEOUT_TMA);
        mbar_wait_bounded(&block_bar, 0);      // give copies in flight one more bounded chance
        return;
    }
    int32_t* W = smem + a.shared_words + warp * a.warp_words;
    uint64_t* bar = reinterpret_cast<uint64_t*>(W + a.warp_words - 4);
    if (lane == 0) mbar_init(bar, 1);
    __syncwarp();
    const long long ntiles = (a.num + a.k - 1) / a.k;
    const long long gw = static_cast<long long>(blockIdx.x) * nwarps + warp;
    const long long nw = static_cast<long long>(gridDim.x) * nwarps;
    unsigned phase = 0;
    for (long long t = gw; t < ntiles; t += nw)
        if (!eval_tile<DM, W16>(a, sh, sp, W, bar, phase, t)) return;
}

// ---------------------------------------------------------------------------
// Streamed form.  No staging pass: each lane reads its own route's op codes
// from global memory through a four-deep register queue (two codes in use,
// the next two loaded at the top of every step, so their latency overlaps
// the step), and checks them as it walks.  A group of G warps walks
// K = floor(32 G / m) candidates at once, lane L of the group taking route
// L mod m of candidate L / m, so for m that does not divide 32 (m = 20: three
// candidates per two warps) candidates straddle warps and far fewer lanes
// idle.  The group meets at a named barrier once per step.  Shared memory
// holds only the ready times, the offsets and a few words per candidate.
//
// Validation without a staging pass.  Offsets are checked first.  Each code
// is range-checked as it is walked.  A drop must find its customer's ready
// slot unresolved (a resolved or picked slot means a second drop: MALFORMED);
// a pickup marks the slot picked (INT32_MIN), so a second pickup of the same
// customer waits forever.  Slots are written by atomic exchange and the old
// value must be the one read: two lanes holding the same op in one step
// cannot both pass.  If every route is walked to its end with no such
// fault, the candidate is a permutation: the n drops are of distinct
// customers, each pickup follows its own customer's drop and no customer is
// picked twice, so the 2n codes hold n drops and n pickups of n distinct
// customers.  A candidate whose walk blocks (a cycle, or a repeated or
// missing op) gets the full check (range and a duplicate bitmap) after the
// walk, which tells MALFORMED from CYCLE.
// ---------------------------------------------------------------------------
constexpr int PICKED = static_cast<int>(0x80000000u);   // ready slot of a customer already picked up

__device__ __forceinline__ void named_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
// barrier of the group plus an OR over its threads' predicates
__device__ __forceinline__ bool named_any(int id, int nthreads, bool pred) {
    unsigned r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(static_cast<unsigned>(pred)), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}

// shared-memory ready slots by 32-bit shared address: a volatile load, and an
// exchange executed only when `on` (else the read value comes back)
__device__ __forceinline__ int lds_volatile(unsigned addr) {
    int v;
    asm volatile("ld.volatile.shared.b32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ int atoms_exch_if(bool on, unsigned addr, int val, int otherwise) {
    int old = otherwise;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %2, 0;\n\t"
        "@p atom.shared.exch.b32 %0, [%1], %3;\n\t}"
        : "+r"(old)
        : "r"(addr), "r"(static_cast<unsigned>(on)), "r"(val)
        : "memory");
    return old;
}

template <int G>
__device__ __forceinline__ void group_sync(int id) {
    if constexpr (G == 1) __syncwarp();
    else named_sync(id, 32 * G);
}
template <int G>
__device__ __forceinline__ bool group_any(int id, bool pred) {
    if constexpr (G == 1) {
        __syncwarp();
        return __any_sync(FULL_MASK, pred) != 0;
    } else {
        return named_any(id, 32 * G, pred);
    }
}

template <int DM, bool W16, int G>
__device__ __forceinline__ void eval_stream_tile(const EvalArgs& a, const int32_t* sh, const int32_t* sp, int32_t* W,
                                                 int gl, int bar_id, long long t) {
    constexpr int NT = 32 * G;
    const int n = a.n, m = a.m, two_n = 2 * n, K = a.K, N1 = n + 1;
    int32_t* ready = W + a.g_ready;     // K x (n+1): -(p+1) unresolved, T_drop + p, or PICKED
    int32_t* soff = W + a.g_off;        // K x (m+1)
    int32_t* flag = W + a.g_flag;       // K: 1 = malformed
    // [2][K]: the last step (of the slot's parity) in which the candidate
    // progressed.  Two slots: a warp of the group that has left step t's
    // barrier may stamp step t+1 before another warp of the group has read
    // step t's stamp; it can never reach step t+2 before that read
    int32_t* prog = W + a.g_prog;
    int32_t* red = W + a.g_red;         // 3 x NT
    const long long first = t * K;
    const int kt = static_cast<int>(min(static_cast<long long>(K), a.num - first));
    const int cand = gl / m, v = gl - cand * m;
    const bool active = cand < kt;

    // ---- 1. offsets, flags, unresolved ready times ----
    for (int i = gl; i < kt * (m + 1); i += NT)
        soff[i] = W16 ? static_cast<int32_t>(__ldg(a.off16 + first * (m + 1) + i)) : __ldg(a.off + first * (m + 1) + i);
    for (int i = gl; i < kt; i += NT) {
        flag[i] = 0;
        prog[i] = -1;
        prog[K + i] = -1;
    }
    for (int g = 0; g < kt; ++g)
        for (int c = gl; c <= n; c += NT) ready[g * N1 + c] = -1 - sp[c];
    group_sync<G>(bar_id);
    // each lane checks the offsets around its route: off[0] = 0, off[m] = 2n, non-decreasing
    int pos = 0, end = 0, start = 0;
    if (active) {
        const int lo = soff[cand * (m + 1) + v], hi = soff[cand * (m + 1) + v + 1];
        if (lo < 0 || hi > two_n || lo > hi || (v == 0 && lo != 0) || (v == m - 1 && hi != two_n)) flag[cand] = 1;
        start = pos = lo;
        end = hi;
    }
    group_sync<G>(bar_id);
    const bool ok_off = active && flag[cand] == 0;

    // ---- 2. the walk (up to two ops per lane per step) ----
    const long long cbase = (first + (active ? cand : 0)) * two_n;
    auto code_at = [&](int q) -> int {
        return W16 ? static_cast<int>(__ldg(a.ops16 + cbase + q)) : __ldg(a.ops + cbase + q);
    };
    // this lane's codes from its current position on, and its candidate's
    // ready slots as a shared-memory address
    const int32_t* rp32 = nullptr;
    const uint16_t* rp16 = nullptr;
    if constexpr (W16) rp16 = a.ops16 + cbase + pos;
    else rp32 = a.ops + cbase + pos;
    const unsigned rdy_addr = smem_u32(ready + (active ? cand : 0) * N1);
    int dep = 0, s = 0, smin = 0, smax = 0, loc = 0;
    bool walking = ok_off && pos < end, cyc = false, bad = false;
    int q0 = walking ? code_at(pos) : 0;
    int q1 = (walking && pos + 1 < end) ? code_at(pos + 1) : 0;
    for (int step = 0;; ++step) {
        int q2 = 0, q3 = 0;
        if (walking && pos + 2 < end) q2 = W16 ? static_cast<int>(__ldg(rp16 + 2)) : __ldg(rp32 + 2);
        if (walking && pos + 3 < end) q3 = W16 ? static_cast<int>(__ldg(rp16 + 3)) : __ldg(rp32 + 3);
        // first op
        const int o1 = walking ? q0 : 0;
        const bool in1 = static_cast<unsigned>(o1 - 2) < static_cast<unsigned>(two_n);
        const int c1 = in1 ? (o1 >> 1) : 0;
        const bool p1 = (o1 & 1) != 0;
        int2 pc1 = make_int2(0, 0);
        int t1;
        if constexpr (DM == VRPRPD_DIST_COORDS) {
            const int2 pl = reinterpret_cast<const int2*>(sh)[loc];
            pc1 = reinterpret_cast<const int2*>(sh)[c1];
            t1 = euc2d_small(pl.x, pl.y, pc1.x, pc1.y);
        } else if constexpr (DM == VRPRPD_DIST_SMEM32 || DM == VRPRPD_DIST_SMEM16) {
            t1 = dist<DM>(a, sh, loc, c1);
        } else {
            t1 = walking ? dist<DM>(a, sh, loc, c1) : 0;
        }
        const unsigned ad1 = rdy_addr + 4u * static_cast<unsigned>(c1);
        const int r1 = lds_volatile(ad1);
        // a drop needs an unresolved slot, -(p+1) in [-2^31 + 1, -1]
        const bool bad1 = walking && (!in1 || (!p1 && static_cast<unsigned>(r1) <= 0x80000000u));
        const bool go1 = walking && !bad1 && (!p1 || r1 >= 0);
        const int a1 = dep + t1;
        // exchange, not store: two lanes that read the same slot in the same
        // step (a repeated op) cannot both see it unchanged
        const int old1 = atoms_exch_if(go1, ad1, p1 ? PICKED : a1 - 1 - r1, r1);
        const bool race1 = old1 != r1;
        dep = go1 ? max(a1, p1 ? r1 : 0) : dep;
        s += go1 ? (p1 ? 1 : -1) : 0;
        smin = min(smin, s);
        smax = max(smax, s);
        pos += go1 ? 1 : 0;
        loc = go1 ? c1 : loc;
        // second op, only behind a first one that went
        const bool try2 = go1 && pos < end;
        const int o2 = try2 ? q1 : 0;
        const bool in2 = static_cast<unsigned>(o2 - 2) < static_cast<unsigned>(two_n);
        const int c2 = in2 ? (o2 >> 1) : 0;
        const bool p2 = (o2 & 1) != 0;
        int t2;
        if constexpr (DM == VRPRPD_DIST_COORDS) {
            const int2 pc2 = reinterpret_cast<const int2*>(sh)[c2];
            t2 = euc2d_small(pc1.x, pc1.y, pc2.x, pc2.y);
        } else if constexpr (DM == VRPRPD_DIST_SMEM32 || DM == VRPRPD_DIST_SMEM16) {
            t2 = dist<DM>(a, sh, c1, c2);
        } else {
            t2 = try2 ? dist<DM>(a, sh, c1, c2) : 0;
        }
        const unsigned ad2 = rdy_addr + 4u * static_cast<unsigned>(c2);
        const int r2 = lds_volatile(ad2);
        const bool bad2 = try2 && (!in2 || (!p2 && static_cast<unsigned>(r2) <= 0x80000000u));
        const bool go2 = try2 && !bad2 && (!p2 || r2 >= 0);
        const int a2 = dep + t2;
        const int old2 = atoms_exch_if(go2, ad2, p2 ? PICKED : a2 - 1 - r2, r2);
        const bool race2 = old2 != r2;
        dep = go2 ? max(a2, p2 ? r2 : 0) : dep;
        s += go2 ? (p2 ? 1 : -1) : 0;
        smin = min(smin, s);
        smax = max(smax, s);
        pos += go2 ? 1 : 0;
        loc = go2 ? c2 : loc;
        // the queue and the code pointer move by the ops taken
        const int took = (go1 ? 1 : 0) + (go2 ? 1 : 0);
        q0 = go2 ? q2 : (go1 ? q1 : q0);
        q1 = go2 ? q3 : (go1 ? q2 : q1);
        if constexpr (W16) rp16 += took;
        else rp32 += took;
        // a repeat caught by the exchange only marks the candidate: the walk
        // goes on (its slots stay in range and it still ends), which keeps the
        // exchange's round trip off the step's critical path
        const bool fault = bad1 || bad2;
        bad = bad || fault || race1 || race2;
        if (go1) prog[(step & 1) * K + cand] = step;
        const bool cont = walking && !fault && pos < end;
        // the group's barrier: every ready time and stamp of this step is
        // visible after it, so a candidate with no progress in a step while
        // unfinished can never progress again (a cycle, or a repeated or
        // missing op that the full check below tells apart)
        const bool any = group_any<G>(bar_id, cont);
        cyc = cyc || (cont && prog[(step & 1) * K + cand] != step);
        walking = cont && !cyc;
        if (!any) break;
    }
    if (bad) flag[cand] = 1;
    if (cyc)                                   // finish the stock prefix of a blocked route
        for (; pos < end; ++pos) {
            const int o = code_at(pos);
            if (o & 1) { ++s; smax = max(smax, s); } else { --s; smin = min(smin, s); }
        }
    red[gl] = cyc ? 1 : 0;
    group_sync<G>(bar_id);

    // ---- 3. full check of the candidates whose walk blocked ----
    for (int g = 0; g < kt; ++g) {
        bool blocked = false;
        for (int j = 0; j < m; ++j) blocked = blocked || red[g * m + j] != 0;
        if (!blocked || flag[g]) continue;     // uniform over the group
        uint32_t* seen = reinterpret_cast<uint32_t*>(ready + g * N1);   // the ready times are no longer needed
        const int sw = (two_n + 2 + 31) / 32;
        for (int i = gl; i < sw; i += NT) seen[i] = 0u;
        group_sync<G>(bar_id);
        const long long gb = (first + g) * two_n;
        for (int e = gl; e < two_n; e += NT) {
            const int o = W16 ? static_cast<int>(__ldg(a.ops16 + gb + e)) : __ldg(a.ops + gb + e);
            bool dup = static_cast<unsigned>(o - 2) >= static_cast<unsigned>(two_n);
            if (!dup) {
                const unsigned bit = 1u << (o & 31);
                dup = (atomicOr(&seen[o >> 5], bit) & bit) != 0u;
            }
            if (dup) flag[g] = 1;
        }
        group_sync<G>(bar_id);
    }

    // ---- 4. per-candidate reduction ----
    int ret = 0, f = 0, pool = 0;
    if (ok_off) {
        if (!cyc && end > start) ret = dep + dist<DM>(a, sh, loc, 0);
        if (a.load_full) {
            f = (smin < -a.Q || smax > 0) ? VRPRPD_VEH_CAP : 0;
            pool = a.Q;
        } else {
            f = (-smin + smax > a.Q) ? VRPRPD_VEH_CAP : 0;
            pool = -smin;
        }
        if (cyc) f |= VRPRPD_CYCLE;
    }
    group_sync<G>(bar_id);                     // the blocked marks above are read
    red[gl] = ret;
    red[NT + gl] = f;
    red[2 * NT + gl] = pool;
    group_sync<G>(bar_id);
    if (active && v == 0) {
        int z = 0, fl = 0;
        long long pl = 0;
        for (int j = 0; j < m; ++j) {
            z = max(z, red[cand * m + j]);
            fl |= red[NT + cand * m + j];
            pl += red[2 * NT + cand * m + j];
        }
        if (pl > a.R) fl |= VRPRPD_POOL;
        if (fl & VRPRPD_CYCLE) z = 0x7fffffff;
        if (flag[cand]) { z = 0x7fffffff; fl = VRPRPD_MALFORMED; }
        a.z[first + cand] = z;
        a.st[first + cand] = static_cast<uint32_t>(fl);
    }
    group_sync<G>(bar_id);                     // the region is reused by the next tile
}

template <int DM, bool W16, int G>
__global__ void __launch_bounds__(1024) eval_stream_kernel(EvalArgs a) {
    extern __shared__ __align__(16) int32_t smem[];
    __shared__ __align__(8) uint64_t block_bar;
    // ---- block-wide staging of the instance (TMA bulk copies) ----
    int32_t* sh = smem;
    int32_t* sp = smem + a.dist_words;
    if (threadIdx.x == 0) {
        mbar_init(&block_bar, 1);
        unsigned dist_bytes = 0;
        if constexpr (DM == VRPRPD_DIST_SMEM32) dist_bytes = ((a.N * a.N * 4) + 15) & ~15;
        if constexpr (DM == VRPRPD_DIST_SMEM16) dist_bytes = ((a.N * a.N * 2) + 15) & ~15;
        if constexpr (DM == VRPRPD_DIST_COORDS) dist_bytes = ((a.N * 8) + 15) & ~15;
        unsigned p_bytes = ((a.N * 4) + 15) & ~15;
        mbar_arrive_expect_tx(&block_bar, dist_bytes + p_bytes);
        if constexpr (DM == VRPRPD_DIST_SMEM32) tma_bulk_g2s(sh, a.d32, dist_bytes, &block_bar);
        if constexpr (DM == VRPRPD_DIST_SMEM16) tma_bulk_g2s(sh, a.d16, dist_bytes, &block_bar);
        if constexpr (DM == VRPRPD_DIST_COORDS) tma_bulk_g2s(sh, a.coords, dist_bytes, &block_bar);
        tma_bulk_g2s(sp, a.p, p_bytes, &block_bar);
    }
    __syncthreads();
    if (!mbar_wait_bounded(&block_bar, 0)) {
        if (threadIdx.x == 0) atomicExch(a.err, DEV_TIMEOUT_TMA);
        mbar_wait_bounded(&block_bar, 0);
        return;
    }
    const int warp = threadIdx.x >> 5, group = warp / G, gl = threadIdx.x - group * 32 * G;
    const int ngroups = (blockDim.x >> 5) / G;
    if (group >= ngroups) return;
    int32_t* W = smem + a.shared_words + static_cast<long long>(group) * a.group_words;
    const long long ntiles = (a.num + a.K - 1) / a.K;
    const long long g0 = static_cast<long long>(blockIdx.x) * ngroups + group;
    const long long ng = static_cast<long long>(gridDim.x) * ngroups;
    for (long long t = g0; t < ntiles; t += ng) eval_stream_tile<DM, W16, G>(a, sh, sp, W, gl, 1 + group, t);
}

// Many instances of uneven size in one persistent launch: tile t of the
// whole job belongs to the instance whose tile prefix brackets it.  Distances
// come from each instance's matrix in global memory (L2-resident); p is read
// through the cache.  Every warp region is sized for the largest instance.
template <int DM>
__global__ void __launch_bounds__(1024) eval_multi_kernel(const EvalArgs* __restrict__ insts,
                                                          const long long* __restrict__ tile_prefix, int n_inst,
                                                          int warp_words) {
    extern __shared__ __align__(16) int32_t smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    int32_t* W = smem + warp * warp_words;
    uint64_t* bar = reinterpret_cast<uint64_t*>(W + warp_words - 4);
    if (lane == 0) mbar_init(bar, 1);
    __syncwarp();
    const long long total = tile_prefix[n_inst];
    const long long gw = static_cast<long long>(blockIdx.x) * nwarps + warp;
    const long long nw = static_cast<long long>(gridDim.x) * nwarps;
    unsigned phase = 0;
    for (long long t = gw; t < total; t += nw) {
        int lo = 0, hi = n_inst;                // prefix[lo] <= t < prefix[lo+1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(tile_prefix + mid) <= t) lo = mid; else hi = mid;
        }
        const EvalArgs a = insts[lo];
        if (!eval_tile<DM, false>(a, nullptr, a.p, W, bar, phase, t - __ldg(tile_prefix + lo))) return;
    }
}


// The same with the streamed walk, one-warp groups: tile t of the whole job is
// ⌊32/m⌋ candidates of the instance whose tile prefix brackets it, walked by
// one warp whose region is sized for the largest instance.
template <int DM>
__global__ void __launch_bounds__(1024) eval_multi_stream_kernel(const EvalArgs* __restrict__ insts,
                                                                 const long long* __restrict__ tile_prefix,
                                                                 int n_inst, int group_words) {
    extern __shared__ __align__(16) int32_t smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    int32_t* W = smem + warp * group_words;
    const long long total = tile_prefix[n_inst];
    const long long gw = static_cast<long long>(blockIdx.x) * nwarps + warp;
    const long long nw = static_cast<long long>(gridDim.x) * nwarps;
    for (long long t = gw; t < total; t += nw) {
        int lo = 0, hi = n_inst;                // prefix[lo] <= t < prefix[lo+1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(tile_prefix + mid) <= t) lo = mid; else hi = mid;
        }
        const EvalArgs a = insts[lo];
        eval_stream_tile<DM, false, 1>(a, nullptr, a.p, W, lane, 0, t - __ldg(tile_prefix + lo));
    }
}

// ---------------------------------------------------------------------------
// Plain form: thread per candidate, global scratch, Kahn order.
// scratch per thread: ready[n+1], pos[m], dep[m], loc[m], seen[(2n+2+31)/32]
// ---------------------------------------------------------------------------
__global__ void eval_plain_kernel(const int32_t* __restrict__ ops, const int32_t* __restrict__ off,
                                  long long num, int n, int m, int R, int Q, int load_full,
                                  const int32_t* __restrict__ d, const int32_t* __restrict__ p,
                                  int32_t* __restrict__ zout, uint32_t* __restrict__ stout,
                                  int32_t* __restrict__ scratch, int scratch_words) {
    const long long tid = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    const long long nthreads = static_cast<long long>(gridDim.x) * blockDim.x;
    const int N = n + 1, two_n = 2 * n, sw = (two_n + 2 + 31) / 32;
    int32_t* ready = scratch + tid * static_cast<long long>(scratch_words);
    int32_t* pos = ready + (n + 1);
    int32_t* dep = pos + m;
    int32_t* loc = dep + m;
    uint32_t* seen = reinterpret_cast<uint32_t*>(loc + m);
    for (long long i = tid; i < num; i += nthreads) {
        const int32_t* o = ops + i * two_n;
        const int32_t* f = off + i * (m + 1);
        uint32_t st = 0;
        if (f[0] != 0 || f[m] != two_n) st = VRPRPD_MALFORMED;
        for (int v = 0; v < m && !st; ++v)
            if (f[v + 1] < f[v]) st = VRPRPD_MALFORMED;
        for (int w = 0; w < sw; ++w) seen[w] = 0u;
        for (int k2 = 0; k2 < two_n && !st; ++k2) {
            const int op = o[k2];
            if (op < 2 || op > two_n + 1) { st = VRPRPD_MALFORMED; break; }
            const uint32_t bit = 1u << (op & 31);
            if (seen[op >> 5] & bit) { st = VRPRPD_MALFORMED; break; }
            seen[op >> 5] |= bit;
        }
        if (st) { zout[i] = 0x7fffffff; stout[i] = st; continue; }
        for (int c = 0; c <= n; ++c) ready[c] = UNRESOLVED;
        for (int v = 0; v < m; ++v) { pos[v] = f[v]; dep[v] = 0; loc[v] = 0; }
        bool progress = true;
        while (progress) {
            progress = false;
            for (int v = 0; v < m; ++v) {
                while (pos[v] < f[v + 1]) {
                    const int op = o[pos[v]], c = op >> 1;
                    const bool pick = op & 1;
                    if (pick && ready[c] < 0) break;
                    const int arr = dep[v] + d[static_cast<long long>(loc[v]) * N + c];
                    if (!pick) { dep[v] = arr; ready[c] = arr + p[c]; }
                    else dep[v] = max(arr, ready[c]);
                    loc[v] = c;
                    ++pos[v];
                    progress = true;
                }
            }
        }
        int z = 0;
        long long pool = 0;
        for (int v = 0; v < m; ++v) {
            if (pos[v] < f[v + 1]) st |= VRPRPD_CYCLE;
            if (f[v + 1] > f[v]) z = max(z, dep[v] + d[static_cast<long long>(loc[v]) * N]);
            int s = 0, smin = 0, smax = 0;
            for (int k2 = f[v]; k2 < f[v + 1]; ++k2) {
                s += (o[k2] & 1) ? 1 : -1;
                smin = min(smin, s);
                smax = max(smax, s);
            }
            if (load_full) {
                if (smin < -Q || smax > 0) st |= VRPRPD_VEH_CAP;
                pool += Q;
            } else {
                if (-smin + smax > Q) st |= VRPRPD_VEH_CAP;
                pool += -smin;
            }
        }
        if (pool > R) st |= VRPRPD_POOL;
        if (st & VRPRPD_CYCLE) z = 0x7fffffff;
        zout[i] = z;
        stout[i] = st;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int round4(long long w) { return static_cast<int>((w + 3) & ~3ll); }

struct Plan {
    int dm = 0, warps = 0, blocks = 0;
    bool w16 = false;    // 16-bit op codes and offsets
    int walk = VRPRPD_WALK_STAGED;
    int G = 1;           // streamed form: warps per group
    size_t smem = 0;
    EvalArgs args{};
};

static bool coords_small(const vrprpd_instance* I) {
    if (!I->has_coords) return false;
    int minx = I->h_coords[0], maxx = minx, miny = I->h_coords[1], maxy = miny;
    for (int i = 0; i <= I->n; ++i) {
        minx = std::min(minx, I->h_coords[2 * i]);
        maxx = std::max(maxx, I->h_coords[2 * i]);
        miny = std::min(miny, I->h_coords[2 * i + 1]);
        maxy = std::max(maxy, I->h_coords[2 * i + 1]);
    }
    long long dx = maxx - minx, dy = maxy - miny;
    return dx * dx + dy * dy < (1ll << 24);
}

bool coords_exact_small(const vrprpd_instance* I) { return coords_small(I); }

bool batched_supported(const vrprpd_instance* I) {
    return I->m <= 32 && 2 * I->n + 1 < (1 << PACK_SHIFT) && I->maxd < (1 << 19);
}

static bool dist_mode_available(const vrprpd_instance* I, int dm) {
    switch (dm) {
        case VRPRPD_DIST_SMEM32: return true;
        case VRPRPD_DIST_SMEM16: return I->has_d16;
        case VRPRPD_DIST_GLOBAL16: return I->has_d16;
        case VRPRPD_DIST_GLOBAL32: return true;
        case VRPRPD_DIST_COORDS: return coords_small(I);
    }
    return false;
}

static bool make_plan(const vrprpd_instance* I, int dm, int warps, int blocks_per_sm, long long num, Plan* P);

// The streamed form's layout: groups of G warps (for G > 1 at most 15 per
// block, one named barrier each), K = floor(32 G / m) candidates per group tile.
static bool make_plan_stream(const vrprpd_instance* I, int dm, int warps, int G, long long num, Plan* P) {
    if (G != 1 && G != 2) return false;
    // groups of more than one warp meet at named barriers 1..15
    if (warps % G != 0 || (G > 1 && warps / G > 15) || 32 * G < I->m) return false;
    if (!make_plan(I, dm, G, 0, num, P)) return false;        // instance words and shared fields
    EvalArgs& a = P->args;
    const long long N1 = I->n + 1;
    a.G = G;
    a.K = (32 * G) / I->m;
    a.g_ready = 0;
    a.g_off = round4(static_cast<long long>(a.K) * N1);
    a.g_flag = a.g_off + round4(static_cast<long long>(a.K) * (I->m + 1));
    a.g_prog = a.g_flag + round4(a.K);
    a.g_red = a.g_prog + round4(2ll * a.K);
    a.group_words = a.g_red + 3 * 32 * G;
    const size_t smem = static_cast<size_t>(a.shared_words + static_cast<long long>(warps / G) * a.group_words) * 4;
    if (smem + 64 > I->smem_optin) return false;
    P->walk = VRPRPD_WALK_STREAMED;
    P->G = G;
    P->warps = warps;
    P->smem = smem;
    return true;
}

// Fill the layout for (dist mode, warps per block); false if it does not fit.
static bool make_plan(const vrprpd_instance* I, int dm, int warps, int blocks_per_sm, long long num, Plan* P) {
    EvalArgs& a = P->args;
    a = EvalArgs{};
    a.n = I->n;
    a.m = I->m;
    a.R = I->R;
    a.Q = I->Q;
    a.N = I->n + 1;
    a.load_full = (I->flags & VRPRPD_LOAD_FULL) != 0;
    a.k = 32 / I->m;
    a.d32 = I->d32;
    a.d16 = I->d16;
    a.coords = I->coords;
    a.p = I->p;
    a.err = I->err;
    a.num = num;
    const long long N = a.N, two_n = 2ll * I->n;
    long long dist_words = 0;
    if (dm == VRPRPD_DIST_SMEM32) dist_words = N * N;
    if (dm == VRPRPD_DIST_SMEM16) dist_words = (N * N + 1) / 2;
    if (dm == VRPRPD_DIST_COORDS) dist_words = 2 * N;
    a.dist_words = round4(dist_words);
    a.shared_words = a.dist_words + round4(N);
    a.sw = static_cast<int>((two_n + 2 + 31) / 32);
    a.a_words = round4((a.k * two_n + 1) / 2 + 2);
    a.ready_words = round4(static_cast<long long>(a.k) * N);
    a.seen_words = round4(static_cast<long long>(a.k) * a.sw);
    a.start_words = 0;
    a.off_words = round4(static_cast<long long>(a.k) * (I->m + 1));
    a.valid_words = round4(a.k);
    a.warp_words = a.a_words + a.ready_words + a.seen_words + a.start_words + a.off_words + a.valid_words + 96 + 4;
    const size_t smem = static_cast<size_t>(a.shared_words + static_cast<long long>(warps) * a.warp_words) * 4;
    if (smem + 64 > I->smem_optin) return false;
    P->dm = dm;
    P->warps = warps;
    P->walk = VRPRPD_WALK_STAGED;
    P->G = 1;
    P->smem = smem;
    return true;
}

template <bool W16, int G>
static const void* stream_kernel_for(int dm) {
    switch (dm) {
        case VRPRPD_DIST_SMEM32: return reinterpret_cast<const void*>(&eval_stream_kernel<VRPRPD_DIST_SMEM32, W16, G>);
        case VRPRPD_DIST_SMEM16: return reinterpret_cast<const void*>(&eval_stream_kernel<VRPRPD_DIST_SMEM16, W16, G>);
        case VRPRPD_DIST_GLOBAL16: return reinterpret_cast<const void*>(&eval_stream_kernel<VRPRPD_DIST_GLOBAL16, W16, G>);
        case VRPRPD_DIST_GLOBAL32: return reinterpret_cast<const void*>(&eval_stream_kernel<VRPRPD_DIST_GLOBAL32, W16, G>);
        default: return reinterpret_cast<const void*>(&eval_stream_kernel<VRPRPD_DIST_COORDS, W16, G>);
    }
}

template <bool W16>
static const void* kernel_for(int dm) {
    switch (dm) {
        case VRPRPD_DIST_SMEM32: return reinterpret_cast<const void*>(&eval_tiles_kernel<VRPRPD_DIST_SMEM32, W16>);
        case VRPRPD_DIST_SMEM16: return reinterpret_cast<const void*>(&eval_tiles_kernel<VRPRPD_DIST_SMEM16, W16>);
        case VRPRPD_DIST_GLOBAL16: return reinterpret_cast<const void*>(&eval_tiles_kernel<VRPRPD_DIST_GLOBAL16, W16>);
        case VRPRPD_DIST_GLOBAL32: return reinterpret_cast<const void*>(&eval_tiles_kernel<VRPRPD_DIST_GLOBAL32, W16>);
        default: return reinterpret_cast<const void*>(&eval_tiles_kernel<VRPRPD_DIST_COORDS, W16>);
    }
}

static const void* plan_kernel(const Plan* P) {
    if (P->walk == VRPRPD_WALK_STREAMED) {
        if (P->G == 2) return P->w16 ? stream_kernel_for<true, 2>(P->dm) : stream_kernel_for<false, 2>(P->dm);
        return P->w16 ? stream_kernel_for<true, 1>(P->dm) : stream_kernel_for<false, 1>(P->dm);
    }
    return P->w16 ? kernel_for<true>(P->dm) : kernel_for<false>(P->dm);
}

static int finalize_plan(const vrprpd_instance* I, int blocks_per_sm, Plan* P) {
    const void* fn = plan_kernel(P);
    { int rc_ = ensure_smem_limit(fn); if (rc_) return rc_; }
    int occ = 0;
    VRP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, P->warps * 32, P->smem));
    VRP_CHECK(occ > 0, VRPRPD_EINVAL, "evaluation layout does not fit on an SM");
    if (blocks_per_sm > 0) occ = std::min(occ, blocks_per_sm);
    const bool streamed = P->walk == VRPRPD_WALK_STREAMED;
    const long long per_tile = streamed ? P->args.K : P->args.k;
    const long long units = streamed ? P->warps / P->G : P->warps;     // tile workers per block
    const long long ntiles = (P->args.num + per_tile - 1) / per_tile;
    long long want = (ntiles + units - 1) / units;
    long long blocks = std::min<long long>(static_cast<long long>(occ) * I->num_sms, want);
    P->blocks = static_cast<int>(std::max<long long>(blocks, 1));
    return VRPRPD_OK;
}

// Default shape: shared-memory distances when they leave room for 8 warps,
// else recomputed coordinates, else L2 gathers.
// host_mapped: the candidates are read in place from pinned host memory over
// the host link, where only the staged walk's coalesced reads are fast; the
// best staged shape the autotuner saw is used then (else the default order).
static int choose_plan(const vrprpd_instance* I, long long num, Plan* P, bool host_mapped = false) {
    EvalTuning T = I->tune;
    if (host_mapped && T.walk != VRPRPD_WALK_STAGED) T = I->tune_staged;
    if (T.dist_mode != VRPRPD_DIST_AUTO && T.warps_per_block > 0) {
        VRP_CHECK(dist_mode_available(I, T.dist_mode), VRPRPD_EINVAL, "configured distance mode unavailable");
        if (T.walk == VRPRPD_WALK_STREAMED) {
            const bool w16 = P->w16;
            VRP_CHECK(make_plan_stream(I, T.dist_mode, T.warps_per_block, T.group_warps, num, P), VRPRPD_EINVAL,
                      "configured streamed layout does not fit (warps %d, group %d)", T.warps_per_block,
                      T.group_warps);
            P->w16 = w16;
            return finalize_plan(I, T.blocks_per_sm, P);
        }
        VRP_CHECK(make_plan(I, T.dist_mode, T.warps_per_block, T.blocks_per_sm, num, P), VRPRPD_EINVAL,
                  "configured evaluation layout exceeds shared memory");
        return finalize_plan(I, T.blocks_per_sm, P);
    }
    const int order[] = {VRPRPD_DIST_SMEM32, VRPRPD_DIST_SMEM16, VRPRPD_DIST_COORDS, VRPRPD_DIST_GLOBAL16,
                         VRPRPD_DIST_GLOBAL32};
    for (int dm : order) {
        if (!dist_mode_available(I, dm)) continue;
        for (int warps : {32, 24, 16, 8}) {
            if (dm != VRPRPD_DIST_GLOBAL32 && dm != VRPRPD_DIST_GLOBAL16 && warps < 8) continue;
            if (make_plan(I, dm, warps, 0, num, P)) return finalize_plan(I, 0, P);
        }
    }
    for (int warps : {8, 4, 2, 1})
        if (make_plan(I, VRPRPD_DIST_GLOBAL32, warps, 0, num, P)) return finalize_plan(I, 0, P);
    set_error("no evaluation layout fits shared memory (n=%d, m=%d)", I->n, I->m);
    return VRPRPD_EINVAL;
}

template <bool W16>
static void launch_tiles(const Plan& P, const EvalArgs& a, cudaStream_t stream) {
    switch (P.dm) {
        case VRPRPD_DIST_SMEM32:
            eval_tiles_kernel<VRPRPD_DIST_SMEM32, W16><<<P.blocks, P.warps * 32, P.smem, stream>>>(a);
            break;
        case VRPRPD_DIST_SMEM16:
            eval_tiles_kernel<VRPRPD_DIST_SMEM16, W16><<<P.blocks, P.warps * 32, P.smem, stream>>>(a);
            break;
        case VRPRPD_DIST_GLOBAL16:
            eval_tiles_kernel<VRPRPD_DIST_GLOBAL16, W16><<<P.blocks, P.warps * 32, P.smem, stream>>>(a);
            break;
        case VRPRPD_DIST_GLOBAL32:
            eval_tiles_kernel<VRPRPD_DIST_GLOBAL32, W16><<<P.blocks, P.warps * 32, P.smem, stream>>>(a);
            break;
        default:
            eval_tiles_kernel<VRPRPD_DIST_COORDS, W16><<<P.blocks, P.warps * 32, P.smem, stream>>>(a);
            break;
    }
}

template <bool W16, int G>
static void launch_stream(const Plan& P, const EvalArgs& a, cudaStream_t stream) {
    const int th = P.warps * 32;
    switch (P.dm) {
        case VRPRPD_DIST_SMEM32: eval_stream_kernel<VRPRPD_DIST_SMEM32, W16, G><<<P.blocks, th, P.smem, stream>>>(a); break;
        case VRPRPD_DIST_SMEM16: eval_stream_kernel<VRPRPD_DIST_SMEM16, W16, G><<<P.blocks, th, P.smem, stream>>>(a); break;
        case VRPRPD_DIST_GLOBAL16: eval_stream_kernel<VRPRPD_DIST_GLOBAL16, W16, G><<<P.blocks, th, P.smem, stream>>>(a); break;
        case VRPRPD_DIST_GLOBAL32: eval_stream_kernel<VRPRPD_DIST_GLOBAL32, W16, G><<<P.blocks, th, P.smem, stream>>>(a); break;
        default: eval_stream_kernel<VRPRPD_DIST_COORDS, W16, G><<<P.blocks, th, P.smem, stream>>>(a); break;
    }
}

static int launch_plan(const Plan& P, cudaStream_t stream) {
    if (P.walk == VRPRPD_WALK_STREAMED) {
        if (P.G == 2) {
            if (P.w16) launch_stream<true, 2>(P, P.args, stream);
            else launch_stream<false, 2>(P, P.args, stream);
        } else {
            if (P.w16) launch_stream<true, 1>(P, P.args, stream);
            else launch_stream<false, 1>(P, P.args, stream);
        }
    } else if (P.w16) {
        launch_tiles<true>(P, P.args, stream);
    } else {
        launch_tiles<false>(P, P.args, stream);
    }
    VRP_CUDA(cudaGetLastError());
    return VRPRPD_OK;
}

static int check_batch(const vrprpd_instance* I, const vrprpd_batch* b, const void* z, const void* st) {
    VRP_CHECK(I && b && z && st, VRPRPD_EINVAL, "NULL argument");
    VRP_CHECK(b->num >= 0, VRPRPD_EINVAL, "negative batch size");
    VRP_CHECK(b->num == 0 || (b->ops && b->off), VRPRPD_EINVAL, "NULL ops/off");
    VRP_CHECK((reinterpret_cast<uintptr_t>(b->ops) & 3u) == 0 && (reinterpret_cast<uintptr_t>(b->off) & 3u) == 0,
              VRPRPD_EINVAL, "ops/off must be 4-byte aligned");
    return VRPRPD_OK;
}

int evaluate_device(const vrprpd_instance* I, const int32_t* ops, const int32_t* off, long long num,
                    int32_t* z, uint32_t* st, cudaStream_t stream, bool host_mapped = false) {
    if (num == 0) return VRPRPD_OK;
    if (!batched_supported(I)) {
        set_error("batched evaluation needs m <= 32, 2n+1 < 4096 and max d < 2^19 (use the plain form)");
        return VRPRPD_EINVAL;
    }
    Plan P;
    int rc = choose_plan(I, num, &P, host_mapped);
    if (rc) return rc;
    P.args.ops = ops;
    P.args.off = off;
    P.args.z = z;
    P.args.st = st;
    return launch_plan(P, stream);
}

// The same evaluation from 16-bit op codes and offsets.
static int evaluate_device16(const vrprpd_instance* I, const uint16_t* ops, const uint16_t* off, long long num,
                             int32_t* z, uint32_t* st, cudaStream_t stream, bool host_mapped = false) {
    if (num == 0) return VRPRPD_OK;
    if (!batched_supported(I)) {
        set_error("batched evaluation needs m <= 32, 2n+1 < 4096 and max d < 2^19 (use the plain form)");
        return VRPRPD_EINVAL;
    }
    Plan P;
    P.w16 = true;
    int rc = choose_plan(I, num, &P, host_mapped);
    if (rc) return rc;
    P.args.ops16 = ops;
    P.args.off16 = off;
    P.args.z = z;
    P.args.st = st;
    return launch_plan(P, stream);
}

static int check_batch16(const vrprpd_instance* I, const vrprpd_batch16* b, const void* z, const void* st) {
    VRP_CHECK(I && b && z && st, VRPRPD_EINVAL, "NULL argument");
    VRP_CHECK(b->num >= 0, VRPRPD_EINVAL, "negative batch size");
    VRP_CHECK(b->num == 0 || (b->ops && b->off), VRPRPD_EINVAL, "NULL ops/off");
    VRP_CHECK((reinterpret_cast<uintptr_t>(b->ops) & 3u) == 0 && (reinterpret_cast<uintptr_t>(b->off) & 1u) == 0,
              VRPRPD_EINVAL, "ops must be 4-byte and off 2-byte aligned");
    return VRPRPD_OK;
}

// Host buffers (ops/off of esz bytes per value): pinned ones are read by the
// kernel in place over the host link (each op is read once, by coalesced
// loads), pageable ones are copied to the device first; the results come back
// to z_host/st_host before the call returns.
static int evaluate_host_impl(vrprpd_instance* I, const void* ops, const void* off, int esz, long long num,
                              int32_t* z_host, uint32_t* st_host, cudaStream_t stream) {
    if (num == 0) return VRPRPD_OK;
    auto run = [&](const void* o, const void* f, int32_t* dz, uint32_t* dst, bool mapped) {
        return esz == 2 ? evaluate_device16(I, static_cast<const uint16_t*>(o), static_cast<const uint16_t*>(f), num,
                                            dz, dst, stream, mapped)
                        : evaluate_device(I, static_cast<const int32_t*>(o), static_cast<const int32_t*>(f), num, dz,
                                          dst, stream, mapped);
    };
    auto grow = [&](size_t need) -> int {
        if (need > I->stage_bytes) {
            if (I->stage) cudaFree(I->stage);
            I->stage = nullptr;
            I->stage_bytes = 0;
            VRP_CUDA(cudaMalloc(&I->stage, need));
            I->stage_bytes = need;
        }
        return VRPRPD_OK;
    };
    const size_t ops_b = static_cast<size_t>(num) * 2 * I->n * esz, off_b = static_cast<size_t>(num) * (I->m + 1) * esz;
    const size_t res_b = (static_cast<size_t>(num) * 4 + 255) & ~static_cast<size_t>(255);
    const void* ops_dev = nullptr;
    const void* off_dev = nullptr;
    {
        cudaPointerAttributes pa{}, pb{};
        if (cudaPointerGetAttributes(&pa, ops) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
            cudaPointerGetAttributes(&pb, off) == cudaSuccess && pb.type == cudaMemoryTypeHost) {
            ops_dev = pa.devicePointer;
            off_dev = pb.devicePointer;
        }
        cudaGetLastError();                    // a pageable pointer is not an error here
    }
    int32_t* d_z;
    int rc;
    if (ops_dev && off_dev) {
        if ((rc = grow(2 * res_b))) return rc;
        d_z = reinterpret_cast<int32_t*>(I->stage);
        rc = run(ops_dev, off_dev, d_z, reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(d_z) + res_b), true);
    } else {
        const size_t ops_r = (ops_b + 255) & ~static_cast<size_t>(255), off_r = (off_b + 255) & ~static_cast<size_t>(255);
        if ((rc = grow(ops_r + off_r + 2 * res_b))) return rc;
        char* base = reinterpret_cast<char*>(I->stage);
        VRP_CUDA(cudaMemcpyAsync(base, ops, ops_b, cudaMemcpyHostToDevice, stream));
        VRP_CUDA(cudaMemcpyAsync(base + ops_r, off, off_b, cudaMemcpyHostToDevice, stream));
        d_z = reinterpret_cast<int32_t*>(base + ops_r + off_r);
        rc = run(base, base + ops_r, d_z, reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(d_z) + res_b), false);
    }
    if (rc) return rc;
    VRP_CUDA(cudaMemcpyAsync(z_host, d_z, num * 4, cudaMemcpyDeviceToHost, stream));
    VRP_CUDA(cudaMemcpyAsync(st_host, reinterpret_cast<char*>(d_z) + res_b, num * 4, cudaMemcpyDeviceToHost, stream));
    VRP_CUDA(cudaStreamSynchronize(stream));
    return VRPRPD_OK;
}

}  // namespace vrp

using namespace vrp;

extern "C" int vrprpd_evaluate(const vrprpd_instance* I, const vrprpd_batch* b, int32_t* z, uint32_t* st,
                               void* stream) {
    int rc = check_batch(I, b, z, st);
    if (rc) return rc;
    return evaluate_device(I, b->ops, b->off, b->num, z, st, static_cast<cudaStream_t>(stream));
}

extern "C" int vrprpd_evaluate_host(const vrprpd_instance* I_, const vrprpd_batch* b, int32_t* z_host,
                                    uint32_t* st_host, void* stream) {
    vrprpd_instance* I = const_cast<vrprpd_instance*>(I_);
    int rc = check_batch(I, b, z_host, st_host);
    if (rc) return rc;
    return evaluate_host_impl(I, b->ops, b->off, 4, b->num, z_host, st_host, static_cast<cudaStream_t>(stream));
}

extern "C" int vrprpd_evaluate16(const vrprpd_instance* I, const vrprpd_batch16* b, int32_t* z, uint32_t* st,
                                 void* stream) {
    int rc = check_batch16(I, b, z, st);
    if (rc) return rc;
    return evaluate_device16(I, b->ops, b->off, b->num, z, st, static_cast<cudaStream_t>(stream));
}

extern "C" int vrprpd_evaluate16_host(const vrprpd_instance* I_, const vrprpd_batch16* b, int32_t* z_host,
                                      uint32_t* st_host, void* stream) {
    vrprpd_instance* I = const_cast<vrprpd_instance*>(I_);
    int rc = check_batch16(I, b, z_host, st_host);
    if (rc) return rc;
    return evaluate_host_impl(I, b->ops, b->off, 2, b->num, z_host, st_host, static_cast<cudaStream_t>(stream));
}

extern "C" int vrprpd_evaluate_plain(const vrprpd_instance* I_, const vrprpd_batch* b, int32_t* z, uint32_t* st,
                                     void* stream) {
    vrprpd_instance* I = const_cast<vrprpd_instance*>(I_);
    int rc = check_batch(I, b, z, st);
    if (rc) return rc;
    if (b->num == 0) return VRPRPD_OK;
    const int threads = 128;
    const long long want = (b->num + threads - 1) / threads;
    const int blocks = static_cast<int>(std::min<long long>(want, 512));
    const int words = (I->n + 1) + 3 * I->m + (2 * I->n + 2 + 31) / 32;
    const size_t need = static_cast<size_t>(blocks) * threads * words;
    if (need > I->plain_scratch_words) {
        cudaFree(I->plain_scratch);
        I->plain_scratch = nullptr;
        I->plain_scratch_words = 0;
        VRP_CUDA(cudaMalloc(&I->plain_scratch, need * 4));
        I->plain_scratch_words = need;
    }
    eval_plain_kernel<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(
        b->ops, b->off, b->num, I->n, I->m, I->R, I->Q, (I->flags & VRPRPD_LOAD_FULL) != 0, I->d32, I->p, z, st,
        I->plain_scratch, words);
    VRP_CUDA(cudaGetLastError());
    return VRPRPD_OK;
}

extern "C" int vrprpd_eval_set_config(vrprpd_instance* I, const vrprpd_eval_config* cfg) {
    VRP_CHECK(I && cfg, VRPRPD_EINVAL, "NULL argument");
    if (cfg->dist_mode == VRPRPD_DIST_AUTO) {
        I->tune = EvalTuning{};
        I->tune_staged = EvalTuning{};
        return VRPRPD_OK;
    }
    VRP_CHECK(cfg->dist_mode >= VRPRPD_DIST_SMEM32 && cfg->dist_mode <= VRPRPD_DIST_COORDS, VRPRPD_EINVAL,
              "bad dist_mode %d", cfg->dist_mode);
    VRP_CHECK(dist_mode_available(I, cfg->dist_mode), VRPRPD_EINVAL, "distance mode %d unavailable here",
              cfg->dist_mode);
    VRP_CHECK(cfg->warps_per_block >= 1 && cfg->warps_per_block <= 32, VRPRPD_EINVAL, "bad warps_per_block");
    VRP_CHECK(cfg->walk == VRPRPD_WALK_STAGED || cfg->walk == VRPRPD_WALK_STREAMED, VRPRPD_EINVAL, "bad walk %d",
              cfg->walk);
    Plan P;
    if (cfg->walk == VRPRPD_WALK_STREAMED) {
        VRP_CHECK(make_plan_stream(I, cfg->dist_mode, cfg->warps_per_block, cfg->group_warps, 1, &P), VRPRPD_EINVAL,
                  "streamed layout does not fit (group_warps must be 1 or 2, divide warps_per_block, leave at "
                  "most 15 groups and cover m lanes)");
    } else {
        VRP_CHECK(make_plan(I, cfg->dist_mode, cfg->warps_per_block, cfg->blocks_per_sm, 1, &P), VRPRPD_EINVAL,
                  "layout exceeds shared memory");
    }
    I->tune.dist_mode = cfg->dist_mode;
    I->tune.warps_per_block = cfg->warps_per_block;
    I->tune.blocks_per_sm = cfg->blocks_per_sm;
    I->tune.walk = cfg->walk;
    I->tune.group_warps = cfg->walk == VRPRPD_WALK_STREAMED ? cfg->group_warps : 1;
    return VRPRPD_OK;
}

extern "C" int vrprpd_eval_get_config(const vrprpd_instance* I, vrprpd_eval_config* cfg) {
    VRP_CHECK(I && cfg, VRPRPD_EINVAL, "NULL argument");
    Plan P;
    int rc = choose_plan(I, 1 << 20, &P);
    if (rc) return rc;
    cfg->dist_mode = P.dm;
    cfg->warps_per_block = P.warps;
    cfg->blocks_per_sm = I->tune.blocks_per_sm;
    cfg->walk = P.walk;
    cfg->group_warps = P.G;
    return VRPRPD_OK;
}

extern "C" int vrprpd_autotune(vrprpd_instance* I, const vrprpd_batch* b, void* stream_, vrprpd_eval_config* chosen) {
    VRP_CHECK(I && b && b->num > 0, VRPRPD_EINVAL, "autotune needs a non-empty batch");
    if (!batched_supported(I)) {
        set_error("batched evaluation unsupported for this instance");
        return VRPRPD_EINVAL;
    }
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    int32_t* z = nullptr;
    uint32_t* st = nullptr;
    VRP_CUDA(cudaMalloc(&z, b->num * 4));
    VRP_CUDA(cudaMalloc(&st, b->num * 4));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 1e30f, best_staged_ms = 1e30f;
    EvalTuning best{}, best_staged{};
    const EvalTuning saved = I->tune;
    const int modes[] = {VRPRPD_DIST_SMEM32, VRPRPD_DIST_SMEM16, VRPRPD_DIST_COORDS, VRPRPD_DIST_GLOBAL16,
                         VRPRPD_DIST_GLOBAL32};
    // the staged walk, then the streamed walk with one- and two-warp groups
    struct Cand { int walk, dm, warps, bps, G; };
    std::vector<Cand> cands;
    for (int dm : modes) {
        if (!dist_mode_available(I, dm)) continue;
        for (int warps : {4, 8, 12, 16, 24, 32})
            for (int bps : {0, 1, 2}) {
                Plan P;
                if (make_plan(I, dm, warps, bps, b->num, &P)) cands.push_back({VRPRPD_WALK_STAGED, dm, warps, bps, 1});
            }
        for (int G : {1, 2})
            for (int warps : {4, 8, 12, 16, 20, 24, 28, 30, 32})
                for (int bps : {0, 1, 2}) {
                    Plan P;
                    if (make_plan_stream(I, dm, warps, G, b->num, &P)) cands.push_back({VRPRPD_WALK_STREAMED, dm, warps, bps, G});
                }
    }
    for (const Cand& cd : cands) {
        I->tune = EvalTuning{cd.dm, cd.warps, cd.bps, cd.walk, cd.G};
        float ms_min = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0, stream);
            int rc = evaluate_device(I, b->ops, b->off, b->num, z, st, stream);
            cudaEventRecord(e1, stream);
            if (rc) break;
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) ms_min = std::min(ms_min, ms);
        }
        if (ms_min < best_ms) {
            best_ms = ms_min;
            best = I->tune;
        }
        if (cd.walk == VRPRPD_WALK_STAGED && ms_min < best_staged_ms) {
            best_staged_ms = ms_min;
            best_staged = I->tune;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(z);
    cudaFree(st);
    if (best.dist_mode == VRPRPD_DIST_AUTO) {
        I->tune = saved;
        set_error("autotune found no runnable configuration");
        return VRPRPD_EINVAL;
    }
    I->tune = best;
    I->tune_staged = best_staged;
    if (chosen) {
        chosen->dist_mode = best.dist_mode;
        chosen->warps_per_block = best.warps_per_block;
        chosen->blocks_per_sm = best.blocks_per_sm;
        chosen->walk = best.walk;
        chosen->group_warps = best.group_warps;
    }
    VRP_CUDA(cudaGetLastError());
    return VRPRPD_OK;
}

// ---------------------------------------------------------------------------
// many instances, one persistent launch
// ---------------------------------------------------------------------------
struct vrprpd_multi {
    int n_inst = 0, device = 0, num_sms = 0;
    size_t smem_optin = 0;
    // per walk (0 staged, 1 streamed): per-instance arguments and tile prefix
    std::vector<EvalArgs> args[2];
    std::vector<long long> prefix[2];
    EvalArgs* d_args[2] = {nullptr, nullptr};
    long long* d_prefix[2] = {nullptr, nullptr};
    int walk = VRPRPD_WALK_STAGED;
    int dm = VRPRPD_DIST_GLOBAL16, warps = 8, blocks = 0, warp_words = 0;
    size_t smem = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t graph_stream = nullptr;
};

namespace vrp {

static const void* multi_kernel(int walk, int dm) {
    if (walk == VRPRPD_WALK_STREAMED)
        return dm == VRPRPD_DIST_GLOBAL16 ? reinterpret_cast<const void*>(&eval_multi_stream_kernel<VRPRPD_DIST_GLOBAL16>)
                                          : reinterpret_cast<const void*>(&eval_multi_stream_kernel<VRPRPD_DIST_GLOBAL32>);
    return dm == VRPRPD_DIST_GLOBAL16 ? reinterpret_cast<const void*>(&eval_multi_kernel<VRPRPD_DIST_GLOBAL16>)
                                      : reinterpret_cast<const void*>(&eval_multi_kernel<VRPRPD_DIST_GLOBAL32>);
}

static int multi_layout(vrprpd_multi* M, int dm, int warps, int walk) {
    const bool streamed = walk == VRPRPD_WALK_STREAMED;
    int ww = 0;
    for (auto& a : M->args[streamed]) ww = std::max(ww, streamed ? a.group_words : a.warp_words);
    const size_t smem = static_cast<size_t>(warps) * ww * 4;
    if (smem + 64 > M->smem_optin) return VRPRPD_EINVAL;
    const void* fn = multi_kernel(walk, dm);
    { int rc_ = ensure_smem_limit(fn); if (rc_) return rc_; }
    int occ = 0;
    VRP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, warps * 32, smem));
    if (occ <= 0) return VRPRPD_EINVAL;
    const long long total = M->prefix[streamed].back();
    M->blocks = static_cast<int>(std::max<long long>(1, std::min<long long>(static_cast<long long>(occ) * M->num_sms,
                                                                         (total + warps - 1) / warps)));
    M->walk = walk;
    M->dm = dm;
    M->warps = warps;
    M->warp_words = ww;
    M->smem = smem;
    if (M->exec) { cudaGraphExecDestroy(M->exec); M->exec = nullptr; }
    if (M->graph) { cudaGraphDestroy(M->graph); M->graph = nullptr; }
    return VRPRPD_OK;
}

static int multi_launch(vrprpd_multi* M, cudaStream_t s) {
    const int w = M->walk == VRPRPD_WALK_STREAMED ? 1 : 0;
    const dim3 grid(M->blocks), block(M->warps * 32);
    if (w && M->dm == VRPRPD_DIST_GLOBAL16)
        eval_multi_stream_kernel<VRPRPD_DIST_GLOBAL16><<<grid, block, M->smem, s>>>(M->d_args[1], M->d_prefix[1],
                                                                                   M->n_inst, M->warp_words);
    else if (w)
        eval_multi_stream_kernel<VRPRPD_DIST_GLOBAL32><<<grid, block, M->smem, s>>>(M->d_args[1], M->d_prefix[1],
                                                                                   M->n_inst, M->warp_words);
    else if (M->dm == VRPRPD_DIST_GLOBAL16)
        eval_multi_kernel<VRPRPD_DIST_GLOBAL16><<<grid, block, M->smem, s>>>(M->d_args[0], M->d_prefix[0],
                                                                            M->n_inst, M->warp_words);
    else
        eval_multi_kernel<VRPRPD_DIST_GLOBAL32><<<grid, block, M->smem, s>>>(M->d_args[0], M->d_prefix[0],
                                                                            M->n_inst, M->warp_words);
    VRP_CUDA(cudaGetLastError());
    return VRPRPD_OK;
}

}  // namespace vrp

extern "C" int vrprpd_multi_create(const vrprpd_instance* const* insts, const vrprpd_batch* batches,
                                   int32_t* const* makespan, uint32_t* const* status, int32_t n_inst,
                                   vrprpd_multi** out) {
    VRP_CHECK(insts && batches && makespan && status && out && n_inst >= 1, VRPRPD_EINVAL, "bad arguments");
    *out = nullptr;
    vrprpd_multi* M = new vrprpd_multi();
    M->n_inst = n_inst;
    M->prefix[0].assign(1, 0);
    M->prefix[1].assign(1, 0);
    bool all16 = true;
    for (int i = 0; i < n_inst; ++i) {
        const vrprpd_instance* I = insts[i];
        int rc = check_batch(I, &batches[i], makespan[i], status[i]);
        if (rc) { delete M; return rc; }
        if (!batched_supported(I)) {
            delete M;
            set_error("instance %d: batched evaluation needs m <= 32, 2n+1 < 4096, max d < 2^19", i);
            return VRPRPD_EINVAL;
        }
        if (i == 0) {
            M->device = I->device;
            M->num_sms = I->num_sms;
            M->smem_optin = I->smem_optin;
        } else if (I->device != M->device) {
            delete M;
            set_error("instances live on different devices");
            return VRPRPD_EINVAL;
        }
        all16 = all16 && I->has_d16;
        // both walks' layouts: the staged one (per warp) and the streamed one
        // (one-warp groups); no instance data is staged in shared memory
        for (int w = 0; w < 2; ++w) {
            Plan P;
            if (w == 0) make_plan(I, VRPRPD_DIST_GLOBAL32, 1, 0, batches[i].num, &P);
            else make_plan_stream(I, VRPRPD_DIST_GLOBAL32, 1, 1, batches[i].num, &P);
            EvalArgs a = P.args;
            a.shared_words = 0;
            a.dist_words = 0;
            a.ops = batches[i].ops;
            a.off = batches[i].off;
            a.z = makespan[i];
            a.st = status[i];
            const long long per_tile = w == 0 ? a.k : a.K;
            M->args[w].push_back(a);
            M->prefix[w].push_back(M->prefix[w].back() + (a.num + per_tile - 1) / per_tile);
        }
    }
    cudaError_t e = cudaSuccess;
    for (int w = 0; w < 2 && e == cudaSuccess; ++w) {
        e = cudaMalloc(&M->d_args[w], sizeof(EvalArgs) * n_inst);
        if (e == cudaSuccess) e = cudaMalloc(&M->d_prefix[w], sizeof(long long) * (n_inst + 1));
        if (e == cudaSuccess)
            e = cudaMemcpy(M->d_args[w], M->args[w].data(), sizeof(EvalArgs) * n_inst, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(M->d_prefix[w], M->prefix[w].data(), sizeof(long long) * (n_inst + 1),
                           cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        set_error("multi_create: %s", cudaGetErrorString(e));
        vrprpd_multi_destroy(M);
        return VRPRPD_ECUDA;
    }
    int rc = VRPRPD_EINVAL;
    for (int warps : {8, 4, 2, 1}) {
        rc = multi_layout(M, all16 ? VRPRPD_DIST_GLOBAL16 : VRPRPD_DIST_GLOBAL32, warps, VRPRPD_WALK_STAGED);
        if (rc == VRPRPD_OK) break;
    }
    if (rc) {
        set_error("multi_create: no layout fits shared memory");
        vrprpd_multi_destroy(M);
        return rc;
    }
    *out = M;
    return VRPRPD_OK;
}

extern "C" int vrprpd_multi_evaluate(vrprpd_multi* M, void* stream_) {
    VRP_CHECK(M, VRPRPD_EINVAL, "NULL plan");
    cudaStream_t s = static_cast<cudaStream_t>(stream_);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (s != nullptr) VRP_CUDA(cudaStreamIsCapturing(s, &cs));
    if (s == nullptr || cs != cudaStreamCaptureStatusNone) return multi_launch(M, s);
    if (!M->exec || M->graph_stream != s) {
        if (M->exec) { cudaGraphExecDestroy(M->exec); M->exec = nullptr; }
        if (M->graph) { cudaGraphDestroy(M->graph); M->graph = nullptr; }
        VRP_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        int rc = multi_launch(M, s);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(s, &g);
        if (rc) { if (g) cudaGraphDestroy(g); return rc; }
        VRP_CHECK(e == cudaSuccess, VRPRPD_ECUDA, "capture failed: %s", cudaGetErrorString(e));
        M->graph = g;
        VRP_CUDA(cudaGraphInstantiate(&M->exec, g, 0));
        M->graph_stream = s;
    }
    VRP_CUDA(cudaGraphLaunch(M->exec, s));
    return VRPRPD_OK;
}

extern "C" int vrprpd_multi_autotune(vrprpd_multi* M, void* stream_, vrprpd_eval_config* chosen) {
    VRP_CHECK(M, VRPRPD_EINVAL, "NULL plan");
    cudaStream_t s = static_cast<cudaStream_t>(stream_);
    bool all16 = true;
    for (auto& a : M->args[0]) all16 = all16 && a.d16 != nullptr;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int bdm = M->dm, bw = M->warps, bwalk = M->walk;
    for (int walk : {VRPRPD_WALK_STAGED, VRPRPD_WALK_STREAMED}) {
        for (int dm : {VRPRPD_DIST_GLOBAL16, VRPRPD_DIST_GLOBAL32}) {
            if (dm == VRPRPD_DIST_GLOBAL16 && !all16) continue;
            for (int warps : {4, 8, 12, 16, 24, 32}) {
                if (multi_layout(M, dm, warps, walk) != VRPRPD_OK) continue;
                float ms_min = 1e30f;
                for (int rep = 0; rep < 3; ++rep) {
                    cudaEventRecord(e0, s);
                    multi_launch(M, s);
                    cudaEventRecord(e1, s);
                    cudaEventSynchronize(e1);
                    float ms = 0;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep > 0) ms_min = std::min(ms_min, ms);
                }
                if (ms_min < best) { best = ms_min; bdm = dm; bw = warps; bwalk = walk; }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int rc = multi_layout(M, bdm, bw, bwalk);
    if (rc) return rc;
    if (chosen) {
        chosen->dist_mode = bdm;
        chosen->warps_per_block = bw;
        chosen->blocks_per_sm = 0;
        chosen->walk = bwalk;
        chosen->group_warps = 1;
    }
    VRP_CUDA(cudaGetLastError());
    return VRPRPD_OK;
}

extern "C" int vrprpd_multi_set_config(vrprpd_multi* M, const vrprpd_eval_config* cfg) {
    VRP_CHECK(M && cfg, VRPRPD_EINVAL, "NULL argument");
    VRP_CHECK(cfg->dist_mode == VRPRPD_DIST_GLOBAL16 || cfg->dist_mode == VRPRPD_DIST_GLOBAL32, VRPRPD_EINVAL,
              "many-instance plans gather distances from L2: dist_mode must be GLOBAL16 or GLOBAL32");
    VRP_CHECK(cfg->walk == VRPRPD_WALK_STAGED || (cfg->walk == VRPRPD_WALK_STREAMED && cfg->group_warps == 1),
              VRPRPD_EINVAL, "walk must be staged, or streamed with one-warp groups");
    if (cfg->dist_mode == VRPRPD_DIST_GLOBAL16)
        for (auto& a : M->args[0]) VRP_CHECK(a.d16 != nullptr, VRPRPD_EINVAL, "an instance has no 16-bit matrix");
    VRP_CHECK(cfg->warps_per_block >= 1 && cfg->warps_per_block <= 32, VRPRPD_EINVAL, "bad warps_per_block");
    const int rc = multi_layout(M, cfg->dist_mode, cfg->warps_per_block, cfg->walk);
    VRP_CHECK(rc == VRPRPD_OK, rc, "this layout does not fit shared memory");
    return VRPRPD_OK;
}

extern "C" void vrprpd_multi_destroy(vrprpd_multi* M) {
    if (!M) return;
    if (M->exec) cudaGraphExecDestroy(M->exec);
    if (M->graph) cudaGraphDestroy(M->graph);
    for (int w = 0; w < 2; ++w) {
        cudaFree(M->d_args[w]);
        cudaFree(M->d_prefix[w]);
    }
    delete M;
}

// ---------------------------------------------------------------------------
// Plain evaluation without any device allocation.
//
// Some callers cannot let the library allocate device memory: code that is
// recording a CUDA graph (an allocation there is not part of the capture and
// breaks it), serving processes that reserve their whole memory budget up
// front and must not grow, and processes whose framework caching allocator
// already holds the free device memory, so a fresh cudaMalloc would fail.
// For them this entry point runs the plain one-thread-per-candidate kernel
// with its per-thread scratch (ready times, route cursors, the op bitmap)
// carved from a fixed array that is part of the library image: 16 MiB on each
// GPU that loads the library, held until the process exits.
// ---------------------------------------------------------------------------
namespace vrp {
constexpr long long NOALLOC_SCRATCH_WORDS = 4ll << 20;   // 4 Mi int32 = 16 MiB
static __device__ __align__(256) int32_t g_noalloc_scratch[NOALLOC_SCRATCH_WORDS];
}  // namespace vrp

extern "C" int vrprpd_evaluate_plain_noalloc_shape(int32_t n, int32_t m, int64_t num, int32_t* blocks,
                                                   int32_t* threads) {
    VRP_CHECK(n >= 1 && m >= 1 && num >= 0 && blocks && threads, VRPRPD_EINVAL, "bad arguments");
    const long long words = (n + 1ll) + 3ll * m + (2ll * n + 2 + 31) / 32;
    const long long max_threads = NOALLOC_SCRATCH_WORDS / words;
    VRP_CHECK(max_threads >= 32, VRPRPD_EINVAL,
              "instance needs %lld scratch words per thread; the fixed %lld-word scratch fits fewer than 32 "
              "threads (use vrprpd_evaluate_plain)", words, NOALLOC_SCRATCH_WORDS);
    // a block of up to 128 threads, a multiple of 32, and only as many
    // blocks as the scratch holds: every launched thread owns its words
    const long long tpb = std::min<long long>(128, max_threads / 32 * 32);
    const long long want = std::max<long long>(1, (num + tpb - 1) / tpb);
    const long long nb = std::max<long long>(1, std::min<long long>(want, max_threads / tpb));
    if (nb * tpb > max_threads) {
        set_error("internal: launch shape exceeds the fixed scratch");
        return VRPRPD_EINVAL;
    }
    *blocks = static_cast<int32_t>(nb);
    *threads = static_cast<int32_t>(tpb);
    return VRPRPD_OK;
}

extern "C" int vrprpd_evaluate_plain_noalloc(const vrprpd_instance* I, const vrprpd_batch* b, int32_t* z,
                                             uint32_t* st, void* stream) {
    int rc = check_batch(I, b, z, st);
    if (rc) return rc;
    if (b->num == 0) return VRPRPD_OK;
    int32_t blocks = 0, threads = 0;
    rc = vrprpd_evaluate_plain_noalloc_shape(I->n, I->m, b->num, &blocks, &threads);
    if (rc) return rc;
    const long long words = (I->n + 1) + 3ll * I->m + (2ll * I->n + 2 + 31) / 32;
    // the array's address on the current device, looked up on every call (the
    // lookup allocates nothing): a cached address would dangle after a
    // device reset reloads the module
    void* scratch = nullptr;
    VRP_CUDA(cudaGetSymbolAddress(&scratch, g_noalloc_scratch));
    eval_plain_kernel<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(
        b->ops, b->off, b->num, I->n, I->m, I->R, I->Q, (I->flags & VRPRPD_LOAD_FULL) != 0, I->d32, I->p, z, st,
        static_cast<int32_t*>(scratch), static_cast<int>(words));
    VRP_CUDA(cudaGetLastError());
    return VRPRPD_OK;
}
