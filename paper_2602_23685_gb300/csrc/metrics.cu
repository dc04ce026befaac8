// Coordination counts of Section 5.2 ("Key Metrics": Cross-Agent % and
// Interleaved %) for a batch of complete solutions of one instance.
//
// One warp per candidate.  A pre-pass over the ops, 32 at a time, checks op
// codes (range, duplicates) and records each customer's dropoff and pickup
// vehicles (a binary search of the op's position in the route offsets).  Then
// lane r walks route r in lock step on the evaluator's semantics (Eqs. 7-12):
// a drop publishes its pickup-ready time, a pickup waits for it and leaves at
// max(arrival, ready).  On the way each lane records, for the customer whose
// dropoff it just made, the arrival at its next op and whether that op is the
// customer's own pickup; each pickup records its completion.  A warp
// reduction over the customers gives
//   cross        dropoff vehicle != pickup vehicle;
//   interleaved  same vehicle: the pickup does not follow its dropoff
//                directly; different vehicles: the dropoff vehicle's next op
//                exists and is reached before the pickup completes.
// A malformed candidate gets -1 for both, a precedence cycle -1 for
// interleaved (its schedule does not exist).
#include <algorithm>

#include "device_common.cuh"
#include "internal.h"

namespace vrp {
namespace {

constexpr int CO_WARPS = 2;
constexpr int NO_NEXT = 0x7fffffff;
constexpr int INFO_DROP_SEEN = 1 << 16, INFO_PICK_SEEN = 1 << 17, INFO_ADJ = 1 << 18;

__host__ __device__ inline int co_stride(int n, int m) { return ((4 * (n + 1) + (m + 1)) + 3) & ~3; }

__global__ void __launch_bounds__(CO_WARPS * 32)
coordination_kernel(const int32_t* __restrict__ ops, const int32_t* __restrict__ off, int num, int n, int m,
                    const int32_t* __restrict__ d, const int32_t* __restrict__ p, int32_t* __restrict__ cross,
                    int32_t* __restrict__ inter) {
    extern __shared__ int co_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int N1 = n + 1, two_n = 2 * n;
    int* base = co_smem + warp * co_stride(n, m);
    volatile int* rdy = base;        // [n+1] pickup-ready time, UNRESOLVED until dropped
    int* na = base + N1;             // [n+1] arrival at the dropoff vehicle's next op
    int* tp = na + N1;               // [n+1] pickup completion
    int* info = tp + N1;             // [n+1] drop vehicle | pickup vehicle << 8 | seen and adjacency bits
    int* F = info + N1;              // [m+1] route offsets
    for (long long i = static_cast<long long>(blockIdx.x) * CO_WARPS + warp; i < num;
         i += static_cast<long long>(gridDim.x) * CO_WARPS) {
        const int32_t* O = ops + i * two_n;
        const int32_t* Fi = off + i * (m + 1);
        for (int c = lane; c <= n; c += 32) {
            rdy[c] = UNRESOLVED;
            na[c] = NO_NEXT;
            tp[c] = 0;
            info[c] = 0;
        }
        for (int v = lane; v <= m; v += 32) F[v] = Fi[v];
        __syncwarp();
        // offsets: 0 = F[0] <= F[1] <= ... <= F[m] = 2n
        bool bad = false;
        for (int v = lane; v < m; v += 32) bad |= F[v] > F[v + 1];
        if (lane == 0) bad |= F[0] != 0 || F[m] != two_n;
        bool anybad = __any_sync(FULL_MASK, bad);
        // ops: in range, no duplicate; vehicles by position
        for (int k0 = 0; k0 < two_n && !anybad; k0 += 32) {
            const int k = k0 + lane;
            if (k < two_n) {
                const int o = O[k];
                if (o < 2 || o > two_n + 1) {
                    bad = true;
                } else {
                    int lo = 0, hi = m;
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (F[mid] <= k) lo = mid; else hi = mid;
                    }
                    const int seen = (o & 1) ? INFO_PICK_SEEN : INFO_DROP_SEEN;
                    const int old = atomicOr(&info[o >> 1], seen | (lo << ((o & 1) ? 8 : 0)));
                    if (old & seen) bad = true;
                }
            }
            anybad = __any_sync(FULL_MASK, bad);
        }
        if (anybad) {
            if (lane == 0) { cross[i] = -1; inter[i] = -1; }
            __syncwarp();
            continue;
        }
        __syncwarp();
        // lock-step walk, one op per lane per step
        const bool mine = lane < m;
        int pos = mine ? F[lane] : 0;
        const int end = mine ? F[lane + 1] : 0;
        int t = 0, loc = 0, prev_drop = 0;
        bool walking = mine && pos < end, cyc = false;
        bool alive = __any_sync(FULL_MASK, walking);
        while (alive) {
            const int o = walking ? O[pos] : 0;
            const int c = o >> 1;
            const bool pick = (o & 1) != 0;
            const int r = (walking && pick) ? rdy[c] : 0;
            const bool go = walking && (!pick || r != UNRESOLVED);
            if (go) {
                const int arr = t + __ldg(d + loc * N1 + c);
                if (prev_drop) na[prev_drop] = arr;
                if (pick) {
                    t = max(arr, r);
                    tp[c] = t;
                    if (prev_drop == c) atomicOr(&info[c], INFO_ADJ);
                    prev_drop = 0;
                } else {
                    t = arr;
                    rdy[c] = arr + __ldg(p + c);
                    prev_drop = c;
                }
                loc = c;
                ++pos;
            }
            const bool more = pos < end;
            const unsigned prog = __ballot_sync(FULL_MASK, go);
            if (walking && more && prog == 0u) cyc = true;
            walking = walking && more && prog != 0u;
            __syncwarp();
            alive = prog != 0u && __any_sync(FULL_MASK, walking);
        }
        const bool anycyc = __any_sync(FULL_MASK, cyc);
        __syncwarp();
        int nc = 0, ni = 0;
        for (int c = 1 + lane; c <= n; c += 32) {
            const int inf = info[c];
            const int vd = inf & 255, vp = (inf >> 8) & 255;
            if (vd != vp) {
                ++nc;
                ni += na[c] < tp[c] ? 1 : 0;
            } else {
                ni += (inf & INFO_ADJ) ? 0 : 1;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            nc += __shfl_xor_sync(FULL_MASK, nc, o);
            ni += __shfl_xor_sync(FULL_MASK, ni, o);
        }
        if (lane == 0) {
            cross[i] = nc;
            inter[i] = anycyc ? -1 : ni;
        }
        __syncwarp();
    }
}

}  // namespace
}  // namespace vrp

using namespace vrp;

extern "C" int vrprpd_coordination(const vrprpd_instance* I, const vrprpd_batch* b, int32_t* cross,
                                   int32_t* interleaved, void* stream) {
    VRP_CHECK(I && b && cross && interleaved, VRPRPD_EINVAL, "NULL argument");
    VRP_CHECK(b->num >= 0, VRPRPD_EINVAL, "negative batch size");
    VRP_CHECK(b->num == 0 || (b->ops && b->off), VRPRPD_EINVAL, "NULL ops/off");
    VRP_CHECK(I->m <= 32, VRPRPD_EINVAL, "coordination counts need m <= 32 (m=%d)", I->m);
    const long long bound = (2ll * I->n + 1) * I->maxd + static_cast<long long>(I->n) * I->maxp;
    VRP_CHECK(bound < (1ll << 31) - 1, VRPRPD_EINVAL, "coordination counts need (2n+1)*max(d) + n*max(p) < 2^31");
    if (b->num == 0) return VRPRPD_OK;
    const size_t smem = static_cast<size_t>(CO_WARPS) * co_stride(I->n, I->m) * sizeof(int);
    VRP_CHECK(smem <= I->smem_optin, VRPRPD_EINVAL, "n=%d too large for the coordination kernel", I->n);
    { int rc_ = ensure_smem_limit(reinterpret_cast<const void*>(&coordination_kernel)); if (rc_) return rc_; }
    int occ = 0;
    VRP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, coordination_kernel, CO_WARPS * 32, smem));
    VRP_CHECK(occ > 0, VRPRPD_EINVAL, "coordination block does not fit on an SM (n=%d)", I->n);
    const long long want = (static_cast<long long>(b->num) + CO_WARPS - 1) / CO_WARPS;
    const int blocks = static_cast<int>(std::min<long long>(want, static_cast<long long>(occ) * I->num_sms));
    coordination_kernel<<<blocks, CO_WARPS * 32, smem, static_cast<cudaStream_t>(stream)>>>(
        b->ops, b->off, b->num, I->n, I->m, I->d32, I->p, cross, interleaved);
    VRP_CUDA(cudaGetLastError());
    return VRPRPD_OK;
}
