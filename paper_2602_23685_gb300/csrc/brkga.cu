// BRKGA on the device (Section 4.4): random-key chromosomes, the multi-pass
// decoder of Algorithm 2, elite preservation, mutants, biased crossover and
// the ALNS warm start (Section 4.4.4).
//
// Per generation (captured once as a CUDA graph, replayed):
//   decode   one warp per chromosome: warp bitonic sort of (key, op index)
//            pairs in shared memory -- the segmented key sort -- then the
//            multi-pass decode with one lane per vehicle; SelectVehicle is a
//            warp argmin of (arrival, vehicle-key rank);
//   evaluate the decoded routes go through the batched evaluator (same
//            makespans by construction; disagreements are counted);
//   rank     one CTA sorts (fitness, index) and records the generation's best;
//   evolve   elites copied, children by biased crossover, mutants drawn.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "device_common.cuh"
#include "internal.h"

namespace vrp {

int evaluate_device(const vrprpd_instance* I, const int32_t* ops, const int32_t* off, long long num, int32_t* z,
                    uint32_t* st, cudaStream_t stream, bool host_mapped = false);
bool batched_supported(const vrprpd_instance* I);

constexpr int DEC_WARPS = 4;
constexpr long long PENALTY = 1000000;

struct BrkgaCtl {
    int gen;            // generation being built
    int sel;            // which key buffer is current
    int mismatches;     // decoder makespan != evaluator makespan (complete decodes)
    int pad;
};

struct DecArgs {
    const float* keys;   // num x L (or two buffers selected by ctl->sel when keys2 != nullptr)
    const float* keys2;
    const BrkgaCtl* ctl;
    int num, n, m, R, Q, load_full, L, P;   // P = power of two >= 2n
    int layout;          // VRPRPD_LAYOUT_VKEYS (2n+m keys) or VRPRPD_LAYOUT_HINTS (4n keys)
    const int32_t* d32;
    const int32_t* p;
    int smem_dist;       // 1 = distance matrix staged in shared memory as int32, 2 = as uint16
    int pack;            // every schedule time is below 2^22: SelectVehicle is one 32-bit reduction
    const uint16_t* d16; // the 16-bit copy (max d < 65536) or null
    int32_t* ops;
    int32_t* off;
    int32_t* z;
    int32_t* unsched;
    long long* fitness;
};

__host__ __device__ inline int pow2_at_least(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

__host__ __device__ inline size_t dec_warp_words(int n, int P) {
    // sort buffer (u64) + tdrop + sched bitmap + per-op (vehicle<<16 | seq) +
    // per-op hinted vehicle (bytes)
    return static_cast<size_t>(2 * P) + (((n + 1) + 3) & ~3) + ((((2 * n + 2 + 31) / 32) + 3) & ~3) +
           (((2 * n) + 3) & ~3) + ((((2 * n + 3) / 4) + 3) & ~3);
}

// The vehicle an assignment hint names: floor(m * alpha) in fp64 (exact for a
// float alpha and m <= 32), capped at m - 1.
__host__ __device__ inline int hint_vehicle(float alpha, int m) {
    const double x = static_cast<double>(alpha) * static_cast<double>(m);
    int h = static_cast<int>(floor(x));
    h = h > m - 1 ? m - 1 : h;
    return h < 0 ? 0 : h;
}

// The decoder specialised on its per-visit choices, so the chain of one op's
// visit holds no branch on them: SD where distances come from (0 L2 int32,
// 1 shared int32, 2 shared uint16), HINTS the 4n layout's tie rule, FULL the
// Eq. 13 start load, PACK the one-reduction SelectVehicle.
template <int SD, bool HINTS, bool FULL, bool PACK>
__global__ void __launch_bounds__(DEC_WARPS * 32, 1) decode_kernel(DecArgs a) {
    extern __shared__ __align__(16) int smem_dec[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = a.n, m = a.m, two_n = 2 * n, N1 = n + 1;
    int* sd = smem_dec;                                   // staged distances (optional)
    const int dist_words = SD == 1 ? ((N1 * N1 + 3) & ~3) : SD == 2 ? (((N1 * N1 + 1) / 2 + 3) & ~3) : 0;
    int* sp = sd + dist_words;
    uint16_t* sd16 = reinterpret_cast<uint16_t*>(sd);
    for (int i = threadIdx.x; i < N1; i += blockDim.x) sp[i] = a.p[i];
    if (SD == 1)
        for (int i = threadIdx.x; i < N1 * N1; i += blockDim.x) sd[i] = a.d32[i];
    if (SD == 2)
        for (int i = threadIdx.x; i < N1 * N1; i += blockDim.x) sd16[i] = a.d16[i];
    int* wbase = sp + ((N1 + 3) & ~3) + warp * static_cast<int>(dec_warp_words(n, a.P));
    unsigned long long* sb = reinterpret_cast<unsigned long long*>(wbase);
    int* tdrop = wbase + 2 * a.P;
    unsigned* sched = reinterpret_cast<unsigned*>(tdrop + (((n + 1) + 3) & ~3));
    int* vs = reinterpret_cast<int*>(sched + ((((two_n + 2 + 31) / 32) + 3) & ~3));
    unsigned char* hv = reinterpret_cast<unsigned char*>(vs + ((two_n + 3) & ~3));
    __syncthreads();
    const float* keys = a.keys;
    if (a.keys2 != nullptr && a.ctl->sel == 1) keys = a.keys2;
    auto dist = [&](int i, int j) -> int {
        if constexpr (SD == 2) return static_cast<int>(sd16[i * N1 + j]);
        else if constexpr (SD == 1) return sd[i * N1 + j];
        else return __ldg(a.d32 + i * N1 + j);
    };
    for (int ch = blockIdx.x * DEC_WARPS + warp; ch < a.num; ch += gridDim.x * DEC_WARPS) {
        const float* kk = keys + static_cast<long long>(ch) * a.L;
        // ---- segmented key sort: (key bits << 32 | op index), padding sorts last ----
        for (int i = lane; i < a.P; i += 32) {
            unsigned long long v = ~0ull;
            if (i < two_n) {
                const float f = __fadd_rn(kk[i], 0.0f);          // -0 -> +0
                v = (static_cast<unsigned long long>(__float_as_uint(f)) << 32) | static_cast<unsigned>(i);
            }
            sb[i] = v;
        }
        for (int i = lane; i <= n; i += 32) tdrop[i] = 0;
        for (int i = lane; i < (two_n + 2 + 31) / 32; i += 32) sched[i] = 0u;
        for (int i = lane; i < two_n; i += 32) vs[i] = -1;
        if (HINTS)
            for (int i = lane; i < two_n; i += 32) hv[i] = static_cast<unsigned char>(hint_vehicle(kk[two_n + i], m));
        __syncwarp();
        for (int size = 2; size <= a.P; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int i = lane; i < a.P / 2; i += 32) {
                    const int lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
                    const bool asc = (lo & size) == 0;
                    const unsigned long long x = sb[lo], y = sb[hi];
                    if ((x > y) == asc) { sb[lo] = y; sb[hi] = x; }
                }
                __syncwarp();
            }
        }
        // ---- tie-break order: vehicle ranks (stable argsort of the m vehicle
        // keys) or, per op, cyclic distance from the hinted vehicle ----
        constexpr bool hints = HINTS;
        const float kv = (!hints && lane < m) ? __fadd_rn(kk[two_n + lane], 0.0f) : 0.0f;
        int rank = 0;
        for (int u = 0; !hints && u < m; ++u) {
            const float ku = __shfl_sync(FULL_MASK, kv, u);
            if (lane < m && (ku < kv || (ku == kv && u < lane))) ++rank;
        }
        // ---- multi-pass decode (Algorithm 2), lane v = vehicle v ----
        int tv = 0, locv = 0, net = 0, nmin = 0, nmax = 0, load = 0, cnt = 0;
        int sum_load = 0, done = 0;
        int len = two_n;                       // sb[0, len): ops not scheduled yet, priority order
        for (int pass = 0; pass < two_n && done < two_n; ++pass) {
            bool progress = false;
            // Whether a drop (a pickup) fits some vehicle does not depend on the
            // customer: it needs one unit of room, resp. stock, on a vehicle.  A
            // drop never makes room for another drop (it lowers its vehicle's
            // stock and raises the pool's load), nor a pickup for another pickup,
            // so once no vehicle takes a drop, every drop fails until a pickup is
            // scheduled, and the other way round.  Those visits are skipped.
            bool drops_blocked = false, picks_blocked = false;
            unsigned long long e_next = len > 0 ? sb[0] : 0ull;
            for (int k = 0; k < len; ++k) {
                // the next op's entry is read ahead: the order does not change
                // within a pass, so its latency overlaps this op
                const unsigned long long e_cur = e_next;
                if (k + 1 < len) e_next = sb[k + 1];
                const int oi = static_cast<int>(e_cur & 0xffffffffu);
                const int o = oi + 2, c = o >> 1;
                const bool pick = (o & 1) != 0;
                // the list holds only ops unscheduled at the pass's start, and only
                // the op visited gets scheduled: o itself is still unscheduled
                if (pick ? picks_blocked : drops_blocked) continue;
                if (pick && !((sched[(2 * c) >> 5] >> ((2 * c) & 31)) & 1u)) continue;
                // the time a pickup waits for, read before the selection
                const int ready = pick ? tdrop[c] + sp[c] : 0;
                bool ok = false;
                if (lane < m) {
                    if (!pick) {
                        if (FULL) ok = net > -a.Q;
                        else {
                            const int nl = max(load, 1 - net);
                            ok = nl + nmax <= a.Q && sum_load - load + nl <= a.R;
                        }
                    } else {
                        ok = FULL ? (net < 0) : (load + net + 1 <= a.Q);
                    }
                }
                const int arr = ok ? tv + dist(locv, c) : 0;
                int tie = rank;
                if (hints) {                       // cyclic distance from the hinted vehicle
                    tie = lane - static_cast<int>(hv[oi]);
                    tie += tie < 0 ? m : 0;
                }
                // SelectVehicle: least arrival, then tie rank, then lane.  With
                // every time below 2^22 the three fit one 32-bit key and one warp
                // reduction; otherwise two reductions
                int win;
                if constexpr (PACK) {
                    const unsigned key = ok ? ((static_cast<unsigned>(arr) << 10) | (static_cast<unsigned>(tie) << 5) |
                                               static_cast<unsigned>(lane))
                                            : 0xffffffffu;
                    const unsigned kmin = __reduce_min_sync(FULL_MASK, key);
                    if (kmin == 0xffffffffu) {
                        if (pick) picks_blocked = true; else drops_blocked = true;
                        continue;
                    }
                    win = static_cast<int>(kmin & 31u);
                } else {
                    const unsigned ua = ok ? static_cast<unsigned>(arr) : 0xffffffffu;
                    const unsigned amin = __reduce_min_sync(FULL_MASK, ua);
                    if (amin == 0xffffffffu) {
                        if (pick) picks_blocked = true; else drops_blocked = true;
                        continue;
                    }
                    const unsigned sub = (ok && ua == amin)
                                             ? ((static_cast<unsigned>(tie) << 5) | static_cast<unsigned>(lane))
                                             : 0xffffffffu;
                    win = static_cast<int>(__reduce_min_sync(FULL_MASK, sub) & 31u);
                }
                // the winner's update, by selects rather than a branch: a drop
                // sets its arrival and lowers the net stock (the start load may
                // grow), a pickup waits for its ready time and raises it
                const bool me = lane == win;
                const int nnet = net + (pick ? 1 : -1);
                const int nnmin = min(nmin, nnet), nnmax = max(nmax, nnet);
                const int nload = pick ? load : -nnmin;
                const int dsum = (me && !pick) ? nload - load : 0;
                if (me) {
                    tv = pick ? max(arr, ready) : arr;
                    net = nnet;
                    nmin = nnmin;
                    nmax = nnmax;
                    load = nload;
                    locv = c;
                    vs[oi] = (lane << 16) | cnt;
                    sched[o >> 5] |= 1u << (o & 31);
                    if (!pick) tdrop[c] = arr;
                }
                // a pickup can make room for drops, a drop stock for pickups
                if (pick) drops_blocked = false; else picks_blocked = false;
                cnt += me ? 1 : 0;
                sum_load += __shfl_sync(FULL_MASK, dsum, win);
                __syncwarp();
                progress = true;
                ++done;
            }
            if (!progress) break;
            // the next pass scans only the ops still unscheduled, order kept (in
            // place: a chunk is read into registers before any of it is written)
            int w = 0;
            for (int base = 0; base < len; base += 32) {
                const int k = base + lane;
                const unsigned long long e = k < len ? sb[k] : 0ull;
                const int o = static_cast<int>(e & 0xffffffffu) + 2;
                const bool keep = k < len && !((sched[o >> 5] >> (o & 31)) & 1u);
                const unsigned bal = __ballot_sync(FULL_MASK, keep);
                __syncwarp();
                if (keep) sb[w + __popc(bal & ((1u << lane) - 1u))] = e;
                w += __popc(bal);
                __syncwarp();
            }
            len = w;
        }
        // ---- outputs: routes, makespan, penalty fitness ----
        int ret = (lane < m && cnt > 0) ? tv + dist(locv, 0) : 0;
        for (int off = 16; off > 0; off >>= 1) ret = max(ret, __shfl_xor_sync(FULL_MASK, ret, off));
        int incl = lane < m ? cnt : 0;
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(FULL_MASK, incl, off);
            if (lane >= off) incl += y;
        }
        const int excl = incl - (lane < m ? cnt : 0);
        int32_t* off_out = a.off + static_cast<long long>(ch) * (m + 1);
        if (lane < m) off_out[lane] = excl;
        if (lane == 0) off_out[m] = done;
        int32_t* ops_out = a.ops + static_cast<long long>(ch) * two_n;
        __syncwarp();
        for (int oi = lane; oi < two_n; oi += 32) {
            const int w = vs[oi];
            if (w < 0) continue;
            const int v = w >> 16, seq = w & 0xffff;
            ops_out[off_out[v] + seq] = oi + 2;
        }
        if (lane == 0) {
            const int un = two_n - done;
            a.z[ch] = ret;
            a.unsched[ch] = un;
            a.fitness[ch] = static_cast<long long>(ret) + PENALTY * un;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// v/m rounded up to the smallest float with m * alpha >= v: the hint that
// hint_vehicle maps back to v
__device__ inline float hint_of(int v, int m) {
    float x = __fdiv_rn(static_cast<float>(v), static_cast<float>(m));
    for (int it = 0; it < 4 && __dmul_rn(static_cast<double>(x), static_cast<double>(m)) < static_cast<double>(v); ++it)
        x = __int_as_float(__float_as_int(x) + 1);
    return x;
}

__global__ void encode_kernel(const int32_t* __restrict__ ops, const int32_t* __restrict__ off, int n, int m,
                              int layout, float* __restrict__ base) {
    // ALNS seed encoding: pi_o = (r-1)/L_v (here r is 0-based); vehicle key
    // v/m, or the hint of vehicle v for each of its ops
    const bool hints = layout == VRPRPD_LAYOUT_HINTS;
    for (int i = threadIdx.x; i < (hints ? 4 * n : 2 * n); i += blockDim.x) base[i] = 0.0f;
    __syncthreads();
    for (int v = 0; v < m; ++v) {
        const int L = off[v + 1] - off[v];
        for (int r = threadIdx.x; r < L; r += blockDim.x) {
            const int oi = ops[off[v] + r] - 2;
            base[oi] = __fdiv_rn(static_cast<float>(r), static_cast<float>(L));
            if (hints) base[2 * n + oi] = hint_of(v, m);
        }
    }
    if (!hints)
        for (int v = threadIdx.x; v < m; v += blockDim.x)
            base[2 * n + v] = __fdiv_rn(static_cast<float>(v), static_cast<float>(m));
}

// Ascending bitonic sort of P (a power of two) keys in shared memory; all
// threads of the block.
static __device__ void seed_sort(unsigned long long* a, int P) {
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

// Construction seeds of the warm start (Section 4.4.4), block h = 0, 1, 2:
// nearest neighbour, load-balanced, shortest processing time.  A customer
// order (the nearest-neighbour tour from the depot; workload 2 d(0,c) + p_c
// descending; p ascending; ties to the smaller id), then every drop before
// every pickup in that order: priority r/(2n) on the r-th drop and (n+r)/(2n)
// on its pickup.  Vehicle part: keys v/m, or hints naming vehicle 0 except
// for the load-balanced seed, whose hints follow a least-loaded assignment in
// its order (ties to the lower index).  out holds 3 chromosomes of L keys.
__global__ void __launch_bounds__(256) seed_kernel(const int32_t* __restrict__ d, const int32_t* __restrict__ p, int n,
                                                   int m, int layout, int L, float* __restrict__ out) {
    extern __shared__ __align__(16) unsigned long long sq[];
    __shared__ unsigned long long wmin[8];
    __shared__ int curc;
    const int h = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int N1 = n + 1;
    int P = 1;
    while (P < n) P <<= 1;
    unsigned char* vis = reinterpret_cast<unsigned char*>(sq + P);
    float* o = out + static_cast<size_t>(h) * L;
    if (h == 0) {
        for (int c = tid; c <= n; c += blockDim.x) vis[c] = 0;
        if (tid == 0) curc = 0;
        __syncthreads();
        for (int r = 0; r < n; ++r) {
            const int cur = curc;
            unsigned long long best = ~0ull;
            for (int c = 1 + tid; c <= n; c += blockDim.x)
                if (!vis[c]) {
                    const unsigned long long k =
                        (static_cast<unsigned long long>(static_cast<unsigned>(__ldg(d + cur * N1 + c))) << 16) |
                        static_cast<unsigned long long>(c);
                    best = k < best ? k : best;
                }
            for (int off = 16; off > 0; off >>= 1) {
                const unsigned long long x = __shfl_xor_sync(0xffffffffu, best, off);
                best = x < best ? x : best;
            }
            if (lane == 0) wmin[warp] = best;
            __syncthreads();
            if (tid == 0) {
                unsigned long long b = wmin[0];
                for (int w = 1; w < static_cast<int>(blockDim.x >> 5); ++w) b = wmin[w] < b ? wmin[w] : b;
                const int c = static_cast<int>(b & 0xFFFF);
                vis[c] = 1;
                sq[r] = static_cast<unsigned long long>(c);
                curc = c;
            }
            __syncthreads();
        }
    } else {
        for (int i = tid; i < P; i += blockDim.x) {
            unsigned long long k = ~0ull;
            if (i < n) {
                const int c = i + 1;
                const long long pc = __ldg(p + c);
                const long long v = h == 1 ? (1ll << 46) - (2ll * __ldg(d + c) + pc) : pc;
                k = (static_cast<unsigned long long>(v) << 16) | static_cast<unsigned long long>(c);
            }
            sq[i] = k;
        }
        seed_sort(sq, P);
    }
    __syncthreads();
    const float two_n = static_cast<float>(2 * n);
    for (int r = tid; r < n; r += blockDim.x) {
        const int c = static_cast<int>(sq[r] & 0xFFFF);
        o[2 * (c - 1)] = __fdiv_rn(static_cast<float>(r), two_n);
        o[2 * (c - 1) + 1] = __fdiv_rn(static_cast<float>(n + r), two_n);
    }
    if (layout != VRPRPD_LAYOUT_HINTS) {
        for (int v = tid; v < m; v += blockDim.x) o[2 * n + v] = __fdiv_rn(static_cast<float>(v), static_cast<float>(m));
    } else if (h != 1) {
        for (int i = tid; i < 2 * n; i += blockDim.x) o[2 * n + i] = hint_of(0, m);
    } else if (warp == 0) {
        long long load = lane < m ? 0 : 0x7fffffffffffffffll;
        for (int r = 0; r < n; ++r) {
            const int c = static_cast<int>(sq[r] & 0xFFFF);
            long long bl = load;
            int bv = lane;
            for (int off = 16; off > 0; off >>= 1) {
                const long long ol = __shfl_xor_sync(0xffffffffu, bl, off);
                const int ov = __shfl_xor_sync(0xffffffffu, bv, off);
                if (ol < bl || (ol == bl && ov < bv)) { bl = ol; bv = ov; }
            }
            if (lane == bv) load += 2ll * __ldg(d + c) + __ldg(p + c);
            if (lane == 0) {
                const float a = hint_of(bv, m);
                o[2 * n + 2 * (c - 1)] = a;
                o[2 * n + 2 * (c - 1) + 1] = a;
            }
        }
    }
}

__global__ void init_pop_kernel(float* __restrict__ keys, const float* __restrict__ base, int pop, int L, int warm,
                                int variants, float eps, unsigned long long key, unsigned long long wkey) {
    const long long total = static_cast<long long>(pop) * L;
    const unsigned long long per = static_cast<unsigned long long>(L) + 2ull;
    const float top = 1.0f - 1.0f / 16777216.0f;
    for (long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; idx < total;
         idx += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int s = static_cast<int>(idx / L), g = static_cast<int>(idx - static_cast<long long>(s) * L);
        float x;
        if (s < warm) {
            // variant 0 is the ALNS encoding itself; with four or more variants
            // the last three perturb the three construction seeds (base + L,
            // + 2L, + 3L), the others the ALNS encoding
            const int nv = variants > 0 ? variants : 1;
            const int var = s % nv;
            const float* bs = base + static_cast<size_t>(nv >= 4 && var >= nv - 3 ? var - (nv - 3) + 1 : 0) * L;
            if (var == 0) {
                x = bs[g];
            } else {
                const float u = draw_key(draw(wkey, static_cast<unsigned long long>(var) * L + g));
                const float e = __fmul_rn(__fsub_rn(__fmul_rn(u, 2.0f), 1.0f), eps);
                x = __fadd_rn(bs[g], e);
                x = x < 0.0f ? 0.0f : x;
                x = x > top ? top : x;
            }
        } else {
            x = draw_key(draw(key, static_cast<unsigned long long>(s) * per + 2ull + g));
        }
        keys[idx] = x;
    }
}

// One CTA: fitness, (fitness, index) sort, generation best.
__global__ void __launch_bounds__(1024) rank_kernel(const int32_t* __restrict__ zdec, const int32_t* __restrict__ un,
                                                    const int32_t* __restrict__ zev, const uint32_t* __restrict__ stev,
                                                    int pop, int P, BrkgaCtl* ctl, int32_t* __restrict__ rank,
                                                    long long* __restrict__ fit, long long* __restrict__ trace) {
    extern __shared__ __align__(16) unsigned long long sk[];
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        unsigned long long v = ~0ull;
        if (i < pop) {
            long long f;
            if (un[i] > 0) {
                f = static_cast<long long>(zdec[i]) + PENALTY * un[i];
            } else {
                f = zev[i];
                if (zev[i] != zdec[i] || stev[i] != 0u) atomicAdd(&ctl->mismatches, 1);
            }
            fit[i] = f;
            v = (static_cast<unsigned long long>(f) << 24) | static_cast<unsigned>(i);
        }
        sk[i] = v;
    }
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < P / 2; i += blockDim.x) {
                const int lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
                const bool asc = (lo & size) == 0;
                const unsigned long long x = sk[lo], y = sk[hi];
                if ((x > y) == asc) { sk[lo] = y; sk[hi] = x; }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < pop; i += blockDim.x) rank[i] = static_cast<int>(sk[i] & 0xffffffu);
    if (threadIdx.x == 0 && trace) trace[ctl->gen] = static_cast<long long>(sk[0] >> 24);
}

// Next population: elites, biased-crossover children, mutants.
__global__ void evolve_kernel(float* __restrict__ buf0, float* __restrict__ buf1, const BrkgaCtl* __restrict__ ctl,
                              const int32_t* __restrict__ rank, int pop, int L, int Ne, int Nc, float rho,
                              unsigned long long key) {
    const float* cur = ctl->sel == 0 ? buf0 : buf1;
    float* nxt = ctl->sel == 0 ? buf1 : buf0;
    const unsigned long long per = static_cast<unsigned long long>(L) + 2ull;
    const unsigned long long gbase = static_cast<unsigned long long>(ctl->gen + 1) * static_cast<unsigned long long>(pop);
    const long long total = static_cast<long long>(pop) * L;
    for (long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; idx < total;
         idx += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int s = static_cast<int>(idx / L), g = static_cast<int>(idx - static_cast<long long>(s) * L);
        float x;
        if (s < Ne) {
            x = cur[static_cast<long long>(rank[s]) * L + g];
        } else {
            const unsigned long long cb = (gbase + static_cast<unsigned long long>(s)) * per;
            if (s < Ne + Nc) {
                const int e = rank[draw_below(draw(key, cb + 0ull), Ne)];
                const int o = rank[Ne + draw_below(draw(key, cb + 1ull), pop - Ne)];
                const float u = draw_key(draw(key, cb + 2ull + g));
                x = u < rho ? cur[static_cast<long long>(e) * L + g] : cur[static_cast<long long>(o) * L + g];
            } else {
                x = draw_key(draw(key, cb + 2ull + g));
            }
        }
        nxt[idx] = x;
    }
}

__global__ void advance_kernel(BrkgaCtl* ctl) {
    ctl->sel ^= 1;
    ctl->gen += 1;
}

// ---------------------------------------------------------------------------
struct DecPlan {
    int blocks = 0, P = 0;
    size_t smem = 0;
    int smem_dist = 0;
};

static int plan_decode(const vrprpd_instance* I, int num, DecPlan* D) {
    VRP_CHECK(I->m <= 32, VRPRPD_EINVAL, "BRKGA decoding needs m <= 32");
    VRP_CHECK(2 * I->n + I->m <= 8192, VRPRPD_EINVAL, "BRKGA decoding needs 2n + m <= 8192");
    const int n = I->n, N1 = n + 1;
    D->P = pow2_at_least(2 * n);
    const size_t warp_words = dec_warp_words(n, D->P);
    const size_t base_words = ((N1 + 3) & ~3) + DEC_WARPS * warp_words;
    // distances staged in shared memory: 16-bit when they fit in that (room for
    // two blocks per SM at n = 200), else 32-bit for small n, else read from L2
    const size_t dist_words32 = (static_cast<size_t>(N1) * N1 + 3) & ~3;
    const size_t dist_words16 = ((static_cast<size_t>(N1) * N1 + 1) / 2 + 3) & ~3;
    size_t dist_words = 0;
    D->smem_dist = 0;
    if (I->has_d16 && (base_words + dist_words16) * 4 + 64 <= I->smem_optin) {
        D->smem_dist = 2;
        dist_words = dist_words16;
    } else if ((base_words + dist_words32) * 4 + 64 <= I->smem_optin && N1 <= 240) {
        D->smem_dist = 1;
        dist_words = dist_words32;
    }
    D->smem = (base_words + dist_words) * 4;
    VRP_CHECK(D->smem + 64 <= I->smem_optin, VRPRPD_EINVAL, "decode shared memory %zu too large", D->smem);
    return VRPRPD_OK;
}

// The decoder instance for these arguments.
template <int SD, bool HINTS, bool FULL>
static const void* decode_fn3(bool pack) {
    return pack ? reinterpret_cast<const void*>(&decode_kernel<SD, HINTS, FULL, true>)
                : reinterpret_cast<const void*>(&decode_kernel<SD, HINTS, FULL, false>);
}
template <int SD>
static const void* decode_fn2(bool hints, bool full, bool pack) {
    if (hints) return full ? decode_fn3<SD, true, true>(pack) : decode_fn3<SD, true, false>(pack);
    return full ? decode_fn3<SD, false, true>(pack) : decode_fn3<SD, false, false>(pack);
}
static const void* decode_fn(int sd, bool hints, bool full, bool pack) {
    if (sd == 2) return decode_fn2<2>(hints, full, pack);
    if (sd == 1) return decode_fn2<1>(hints, full, pack);
    return decode_fn2<0>(hints, full, pack);
}
static const void* decode_fn(const DecArgs& a) {
    return decode_fn(a.smem_dist, a.layout == VRPRPD_LAYOUT_HINTS, a.load_full != 0, a.pack != 0);
}
// The grid of the instance that decodes with arguments a: as many blocks as
// the chromosomes need, at most what stays resident on all SMs.
static int plan_decode_grid(const vrprpd_instance* I, int num, const DecArgs& a, DecPlan* D) {
    const void* fn = decode_fn(a);
    { int rc_ = ensure_smem_limit(fn); if (rc_) return rc_; }
    int occ = 0;
    VRP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, DEC_WARPS * 32, D->smem));
    VRP_CHECK(occ > 0, VRPRPD_EINVAL, "decode block does not fit");
    D->blocks = std::max(1, std::min((num + DEC_WARPS - 1) / DEC_WARPS, occ * I->num_sms));
    return VRPRPD_OK;
}
static cudaError_t launch_decode(const DecArgs& a, int blocks, size_t smem, cudaStream_t s) {
    DecArgs args = a;
    void* params[] = {&args};
    return cudaLaunchKernel(decode_fn(a), dim3(blocks), dim3(DEC_WARPS * 32), params, smem, s);
}

static DecArgs dec_args(const vrprpd_instance* I, const DecPlan& D, int num, int layout) {
    DecArgs a{};
    a.num = num;
    a.n = I->n;
    a.m = I->m;
    a.R = I->R;
    a.Q = I->Q;
    a.load_full = (I->flags & VRPRPD_LOAD_FULL) != 0;
    a.layout = layout;
    a.L = layout == VRPRPD_LAYOUT_HINTS ? 4 * I->n : 2 * I->n + I->m;
    a.P = D.P;
    a.d32 = I->d32;
    a.p = I->p;
    a.smem_dist = D.smem_dist;
    a.d16 = I->d16;
    // a decoded schedule is a precedence graph of the instance's ops, so no
    // time exceeds (2n+1) max d + n max p
    const long long bound = (2ll * I->n + 1) * I->maxd + static_cast<long long>(I->n) * I->maxp;
    a.pack = bound < (1ll << 22) && I->m <= 32 ? 1 : 0;
    return a;
}

}  // namespace vrp

using namespace vrp;

extern "C" void vrprpd_brkga_params_default(vrprpd_brkga_params* P) {
    if (!P) return;
    P->pop = 30000;
    P->generations = 20000;
    P->warm_slots = -1;        // ceil(0.15 * pop), worked out by vrprpd_brkga_run
    P->warm_variants = 20;
    P->elite_frac = 0.15f;
    P->mutant_frac = 0.15f;
    P->rho = 0.7f;
    P->eps = 0.03f;
    P->layout = VRPRPD_LAYOUT_VKEYS;
}

extern "C" int vrprpd_brkga_decode(const vrprpd_instance* I, const float* keys, int32_t num, int32_t layout,
                                   int32_t* ops, int32_t* off, int32_t* z, int32_t* unsched, int64_t* fitness,
                                   void* stream) {
    VRP_CHECK(I && keys && ops && off && z && unsched && fitness, VRPRPD_EINVAL, "NULL argument");
    VRP_CHECK(num >= 0, VRPRPD_EINVAL, "negative count");
    VRP_CHECK(layout == VRPRPD_LAYOUT_VKEYS || layout == VRPRPD_LAYOUT_HINTS, VRPRPD_EINVAL, "unknown key layout %d",
              layout);
    if (num == 0) return VRPRPD_OK;
    DecPlan D;
    int rc = plan_decode(I, num, &D);
    if (rc) return rc;
    DecArgs a = dec_args(I, D, num, layout);
    rc = plan_decode_grid(I, num, a, &D);
    if (rc) return rc;
    a.keys = keys;
    a.ops = ops;
    a.off = off;
    a.z = z;
    a.unsched = unsched;
    a.fitness = reinterpret_cast<long long*>(fitness);
    VRP_CUDA(launch_decode(a, D.blocks, D.smem, static_cast<cudaStream_t>(stream)));
    return VRPRPD_OK;
}

extern "C" int vrprpd_brkga_run(const vrprpd_instance* I, const vrprpd_brkga_params* P, const vrprpd_solution* warm,
                                uint64_t seed, vrprpd_solution* best, int64_t* best_fitness, int64_t* trace,
                                float* final_keys, void* stream_) {
    VRP_CHECK(I && P && best && best->ops && best->off, VRPRPD_EINVAL, "NULL argument");
    VRP_CHECK(P->pop >= 2 && P->pop <= 16384, VRPRPD_EINVAL, "pop must lie in [2, 16384]");
    VRP_CHECK(P->generations >= 1, VRPRPD_EINVAL, "generations must be >= 1");
    VRP_CHECK(batched_supported(I), VRPRPD_EINVAL, "the batched evaluator does not support this instance");
    VRP_CHECK(P->layout == VRPRPD_LAYOUT_VKEYS || P->layout == VRPRPD_LAYOUT_HINTS, VRPRPD_EINVAL,
              "unknown key layout %d", P->layout);
    const int n = I->n, m = I->m, pop = P->pop, G = P->generations;
    const int L = P->layout == VRPRPD_LAYOUT_HINTS ? 4 * n : 2 * n + m;
    int Ne = static_cast<int>(std::floor(static_cast<double>(P->elite_frac) * pop));
    int Nm = static_cast<int>(std::floor(static_cast<double>(P->mutant_frac) * pop));
    if (Ne < 1) Ne = 1;
    if (Ne + Nm > pop) Nm = pop - Ne;
    const int Nc = pop - Ne - Nm;
    // a negative count asks for Section 4.4.4's 15% of the population, rounded up
    const int warm_req = P->warm_slots < 0 ? static_cast<int>((15ll * pop + 99) / 100) : P->warm_slots;
    const int warm_slots = warm ? std::min(warm_req, pop) : 0;
    // work already queued on the caller's stream comes first
    VRP_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream_)));
    cudaStream_t s;
    VRP_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    // device buffers
    const size_t keys_b = static_cast<size_t>(pop) * L * 4;
    std::vector<void*> allocs;
    bool alloc_failed = false;
    auto dalloc = [&](size_t bytes) -> void* {
        void* p = nullptr;
        if (cudaMallocAsync(&p, std::max<size_t>(bytes, 16), s) != cudaSuccess) {
            alloc_failed = true;
            return nullptr;
        }
        allocs.push_back(p);
        return p;
    };
    auto cleanup = [&]() {
        for (void* p : allocs) cudaFreeAsync(p, s);
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    };
    float* buf0 = static_cast<float*>(dalloc(keys_b));
    float* buf1 = static_cast<float*>(dalloc(keys_b));
    float* base = static_cast<float*>(dalloc(static_cast<size_t>(4) * L * 4));   // ALNS encoding + 3 seeds
    int32_t* dops = static_cast<int32_t*>(dalloc(static_cast<size_t>(pop) * 2 * n * 4));
    int32_t* doff = static_cast<int32_t*>(dalloc(static_cast<size_t>(pop) * (m + 1) * 4));
    int32_t* zdec = static_cast<int32_t*>(dalloc(pop * 4));
    int32_t* un = static_cast<int32_t*>(dalloc(pop * 4));
    long long* fitd = static_cast<long long*>(dalloc(pop * 8));
    int32_t* zev = static_cast<int32_t*>(dalloc(pop * 4));
    uint32_t* stev = static_cast<uint32_t*>(dalloc(pop * 4));
    int32_t* rank = static_cast<int32_t*>(dalloc(pop * 4));
    long long* fit = static_cast<long long*>(dalloc(pop * 8));
    long long* dtrace = static_cast<long long*>(dalloc(static_cast<size_t>(G) * 8));
    BrkgaCtl* ctl = static_cast<BrkgaCtl*>(dalloc(sizeof(BrkgaCtl)));
    int32_t* wops = static_cast<int32_t*>(dalloc(2 * n * 4));
    int32_t* woff = static_cast<int32_t*>(dalloc((m + 1) * 4));
    if (alloc_failed) { cleanup(); set_error("BRKGA: device allocation failed"); return VRPRPD_ENOMEM; }
    const unsigned long long key = stream_key(seed, RNG_STREAM_BRKGA), wkey = stream_key(seed, RNG_STREAM_WARM);
    BrkgaCtl c0{0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(ctl, &c0, sizeof(c0), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(base, 0, static_cast<size_t>(4) * L * 4, s);
    if (warm && e == cudaSuccess) {
        e = cudaMemcpyAsync(wops, warm->ops, 2 * n * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(woff, warm->off, (m + 1) * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) encode_kernel<<<1, 256, 0, s>>>(wops, woff, n, m, P->layout, base);
        if (e == cudaSuccess) {
            int Ps = 1;
            while (Ps < n) Ps <<= 1;
            seed_kernel<<<3, 256, static_cast<size_t>(Ps) * 8 + n + 16, s>>>(I->d32, I->p, n, m, P->layout, L,
                                                                          base + L);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) {
        init_pop_kernel<<<std::min<long long>((static_cast<long long>(pop) * L + 255) / 256, 4096), 256, 0, s>>>(
            buf0, base, pop, L, warm_slots, P->warm_variants, P->eps, key, wkey);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) { cleanup(); set_error("BRKGA init: %s", cudaGetErrorString(e)); return VRPRPD_ECUDA; }
    DecPlan D;
    int rc = plan_decode(I, pop, &D);
    if (rc) { cleanup(); return rc; }
    DecArgs da = dec_args(I, D, pop, P->layout);
    rc = plan_decode_grid(I, pop, da, &D);
    if (rc) { cleanup(); return rc; }
    da.keys = buf0;
    da.keys2 = buf1;
    da.ctl = ctl;
    da.ops = dops;
    da.off = doff;
    da.z = zdec;
    da.unsched = un;
    da.fitness = fitd;
    const int Prank = pow2_at_least(pop);
    const size_t rank_smem = static_cast<size_t>(Prank) * 8;
    VRP_CHECK(rank_smem + 64 <= I->smem_optin, VRPRPD_EINVAL, "population too large for the ranking kernel");
    { int rc_ = ensure_smem_limit(reinterpret_cast<const void*>(&rank_kernel)); if (rc_) { cleanup(); return rc_; } }
    const int evo_blocks = static_cast<int>(std::min<long long>((static_cast<long long>(pop) * L + 255) / 256, 8192));
    auto enqueue_eval_rank = [&]() -> int {
        VRP_CUDA(launch_decode(da, D.blocks, D.smem, s));
        int r = evaluate_device(I, dops, doff, pop, zev, stev, s);
        if (r) return r;
        rank_kernel<<<1, 1024, rank_smem, s>>>(zdec, un, zev, stev, pop, Prank, ctl, rank, fit, dtrace);
        VRP_CUDA(cudaGetLastError());
        return VRPRPD_OK;
    };
    // warm-up pass outside capture so every kernel attribute is set
    rc = VRPRPD_OK;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (G > 1) {
        VRP_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        rc = enqueue_eval_rank();
        if (rc == VRPRPD_OK) {
            evolve_kernel<<<evo_blocks, 256, 0, s>>>(buf0, buf1, ctl, rank, pop, L, Ne, Nc, P->rho, key);
            advance_kernel<<<1, 1, 0, s>>>(ctl);
        }
        cudaError_t ce = cudaStreamEndCapture(s, &graph);
        if (rc == VRPRPD_OK && ce != cudaSuccess) { set_error("graph capture: %s", cudaGetErrorString(ce)); rc = VRPRPD_ECUDA; }
        if (rc == VRPRPD_OK) {
            ce = cudaGraphInstantiate(&exec, graph, 0);
            if (ce != cudaSuccess) { set_error("graph instantiate: %s", cudaGetErrorString(ce)); rc = VRPRPD_ECUDA; }
        }
        for (int g = 0; rc == VRPRPD_OK && g < G - 1; ++g) {
            ce = cudaGraphLaunch(exec, s);
            if (ce != cudaSuccess) { set_error("graph launch: %s", cudaGetErrorString(ce)); rc = VRPRPD_ECUDA; }
        }
    }
    if (rc == VRPRPD_OK) rc = enqueue_eval_rank();          // last generation: evaluate and rank only
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (rc) { cleanup(); return rc; }
    e = cudaStreamSynchronize(s);
    BrkgaCtl cend{};
    int best_idx = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&cend, ctl, sizeof(cend), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&best_idx, rank, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    long long bf = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bf, fit + best_idx, 8, cudaMemcpyDeviceToHost, s);
    int32_t bz = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(best->ops, dops + static_cast<long long>(best_idx) * 2 * n, 2 * n * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(best->off, doff + static_cast<long long>(best_idx) * (m + 1), (m + 1) * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bz, zdec + best_idx, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && trace) e = cudaMemcpyAsync(trace, dtrace, static_cast<size_t>(G) * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && final_keys)
        e = cudaMemcpyAsync(final_keys, cend.sel == 0 ? buf0 : buf1, keys_b, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { cleanup(); set_error("BRKGA copy-out: %s", cudaGetErrorString(e)); return VRPRPD_ECUDA; }
    best->makespan = bz;
    best->status = 0;
    if (best_fitness) *best_fitness = bf;
    cleanup();
    if (cend.mismatches != 0) {
        set_error("BRKGA: %d decoded makespans disagree with the evaluator", cend.mismatches);
        return VRPRPD_ECUDA;
    }
    return VRPRPD_OK;
}
