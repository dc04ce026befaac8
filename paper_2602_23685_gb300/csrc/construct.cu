// The paper's three-phase initial solution (Section 4.2.5), one CTA:
//   1. sweep: customers by exact angle around the depot (half plane, then
//      the integer cross product, then id; by id without coordinates), a
//      bitonic sort with that comparison; cut into m' = min(m, R) sectors of
//      equal count (customer k of the order in sector floor(k m' / n));
//   2. load balancing on w_c = 2 d(0,c) + p_c (one thread): while the spread
//      of the sector workloads is 10% of their mean or more, the heaviest
//      sector (lowest index on ties) hands its boundary customer to its
//      lighter neighbour (lower index on ties), unless that would leave the
//      neighbour at least as heavy as the heaviest was; at most 4n moves;
//   3. nearest-neighbour routes (one thread per vehicle): vehicle v serves
//      its sector alone from the depot at time 0 with b = min(Q, floor(R/m'))
//      resources, each step taking the feasible op that completes first (a
//      drop while a resource is left: its arrival; a pickup of a dropped
//      customer: max(arrival, T_drop + p)), ties by travel, then drop before
//      pickup, then op code.
// Vehicle v's ops start at 2 * (first customer index of its sector), so the
// route offsets follow from the sector bounds.  The refinement rounds that
// follow run in the ALNS kernel's local search.
#include <algorithm>

#include "device_common.cuh"
#include "internal.h"

namespace vrp {
namespace {

__device__ __forceinline__ bool angle_before(const int32_t* xy, int a, int b) {
    const long long ax = xy[2 * a] - xy[0], ay = xy[2 * a + 1] - xy[1];
    const long long bx = xy[2 * b] - xy[0], by = xy[2 * b + 1] - xy[1];
    const int ha = (ay < 0 || (ay == 0 && ax < 0)) ? 1 : 0, hb = (by < 0 || (by == 0 && bx < 0)) ? 1 : 0;
    if (ha != hb) return ha < hb;
    const long long cr = ax * by - ay * bx;
    if (cr != 0) return cr > 0;
    return a < b;
}

__global__ void __launch_bounds__(256) construct_kernel(const int32_t* __restrict__ xy, const int32_t* __restrict__ d,
                                                        const int32_t* __restrict__ p, int n, int m, int R, int Q,
                                                        int32_t* __restrict__ ops, int32_t* __restrict__ off) {
    extern __shared__ __align__(16) long long csm[];
    __shared__ int start[33];
    __shared__ long long Wl[32];
    const int tid = threadIdx.x, N1 = n + 1;
    int P = 1;
    while (P < n) P <<= 1;
    long long* rdy = csm;                                        // [n+1]
    int* ord = reinterpret_cast<int*>(rdy + N1);                 // [P]
    unsigned char* state = reinterpret_cast<unsigned char*>(ord + P);   // [n+1]
    const int mp = m < R ? m : R;
    const int b = min(Q, R / mp);
    // 1. sweep order (entries past n sort last)
    for (int i = tid; i < P; i += blockDim.x) ord[i] = i < n ? i + 1 : 0x7fffffff;
    for (int c = tid; c <= n; c += blockDim.x) { state[c] = 0; rdy[c] = 0; }
    __syncthreads();
    if (xy) {
        for (int size = 2; size <= P; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int i = tid; i < P / 2; i += blockDim.x) {
                    const int lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
                    const bool asc = (lo & size) == 0;
                    const int x = ord[lo], y = ord[hi];
                    const bool y_first = y != 0x7fffffff && (x == 0x7fffffff || angle_before(xy, y, x));
                    if (y_first == asc) { ord[lo] = y; ord[hi] = x; }
                }
                __syncthreads();
            }
        }
    }
    // 2. sectors and load balancing
    if (tid == 0) {
        for (int s = 0; s < mp; ++s) Wl[s] = 0;
        for (int k = 0; k < n; ++k) {
            const int s = static_cast<int>((static_cast<long long>(k) * mp) / n);
            const int c = ord[k];
            Wl[s] += 2ll * __ldg(d + c) + __ldg(p + c);
        }
        for (int s = 0; s <= mp; ++s) start[s] = static_cast<int>((static_cast<long long>(s) * n + mp - 1) / mp);
        for (int mv = 0; mv < 4 * n && mp > 1; ++mv) {
            int h = 0, l = 0;
            long long tot = 0;
            for (int s = 0; s < mp; ++s) {
                tot += Wl[s];
                if (Wl[s] > Wl[h]) h = s;
                if (Wl[s] < Wl[l]) l = s;
            }
            if (10ll * mp * (Wl[h] - Wl[l]) < tot) break;
            int g = -1;
            if (h > 0) g = h - 1;
            if (h + 1 < mp && (g < 0 || Wl[h + 1] < Wl[g])) g = h + 1;
            if (start[h + 1] == start[h]) break;
            const int c = g < h ? ord[start[h]] : ord[start[h + 1] - 1];
            const long long wc = 2ll * __ldg(d + c) + __ldg(p + c);
            if (Wl[g] + wc >= Wl[h]) break;
            Wl[g] += wc;
            Wl[h] -= wc;
            if (g < h) start[h] += 1; else start[h + 1] -= 1;
        }
    }
    __syncthreads();
    // 3. nearest-neighbour routes, one thread per vehicle
    if (tid < mp) {
        const int v = tid, k0 = start[v], k1 = start[v + 1];
        long long t = 0;
        int loc = 0, out = 0, w = 2 * k0;
        for (int step = 0; step < 2 * (k1 - k0); ++step) {
            int bo = -1;
            long long bt = 0, bd = 0;
            for (int k = k0; k < k1; ++k) {
                const int c = ord[k];
                const int st = state[c];
                if (st == 2 || (st == 0 && out >= b)) continue;
                const int pick = st == 1 ? 1 : 0;
                const long long dl = __ldg(d + loc * N1 + c);
                long long fin = t + dl;
                if (pick && rdy[c] > fin) fin = rdy[c];
                const int o = 2 * c + pick;
                bool better = bo < 0;
                if (!better) {
                    if (fin != bt) better = fin < bt;
                    else if (dl != bd) better = dl < bd;
                    else if ((o & 1) != (bo & 1)) better = (o & 1) < (bo & 1);
                    else better = o < bo;
                }
                if (better) { bo = o; bt = fin; bd = dl; }
            }
            const int c = bo >> 1;
            if (bo & 1) { state[c] = 2; --out; }
            else { state[c] = 1; ++out; rdy[c] = bt + __ldg(p + c); }
            t = bt;
            loc = c;
            ops[w++] = bo;
        }
    }
    for (int v = tid; v <= m; v += blockDim.x) off[v] = v <= mp ? 2 * start[v] : 2 * n;
}

}  // namespace

// Launch the constructor into device buffers ops (2n) and off (m+1).
int construct_paper_device(const vrprpd_instance* I, int32_t* ops, int32_t* off, cudaStream_t stream) {
    VRP_CHECK(I->R >= 1 && I->Q >= 1, VRPRPD_EINVAL, "initial solution needs R >= 1 and Q >= 1");
    VRP_CHECK(I->m <= 32, VRPRPD_EINVAL, "the three-phase constructor needs m <= 32");
    const int n = I->n;
    int P = 1;
    while (P < n) P <<= 1;
    const size_t smem = static_cast<size_t>(n + 1) * 8 + static_cast<size_t>(P) * 4 + n + 1 + 16;
    VRP_CHECK(smem <= I->smem_optin, VRPRPD_EINVAL, "n=%d too large for the constructor", n);
    { int rc_ = ensure_smem_limit(reinterpret_cast<const void*>(&construct_kernel)); if (rc_) return rc_; }
    construct_kernel<<<1, 256, smem, stream>>>(I->has_coords ? I->coords : nullptr, I->d32, I->p, n, I->m, I->R,
                                               I->Q, ops, off);
    VRP_CUDA(cudaGetLastError());
    return VRPRPD_OK;
}

}  // namespace vrp
