// Device helpers: TMA bulk copies and mbarriers (inline PTX), exact EUC_2D,
// the counter-based RNG and the acceptance-test exp.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace vrp {

constexpr unsigned FULL_MASK = 0xffffffffu;
constexpr int UNRESOLVED = -1;            // ready time of a customer not yet dropped
constexpr int PACK_SHIFT = 12;            // packed op word: (travel-in << 12) | op code
constexpr int PACK_MASK = (1 << PACK_SHIFT) - 1;
constexpr long long MBAR_SPIN_LIMIT = 1ll << 24;

// ---------------------------------------------------------------------------
// mbarrier + cp.async.bulk (TMA bulk copy global -> shared, non-multicast)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// try_wait with a suspend-time hint (ns): the waiting thread sleeps instead of
// spinning, so other warps get the issue slots.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(1000000u)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait: true when the phase completed, false after ~2 s or the spin
// limit, whichever comes first.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
    const uint64_t t0 = global_ns();
    for (long long i = 0; i < MBAR_SPIN_LIMIT; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > 2000000000ull) return false;
    }
    return false;
}

// Order this thread's generic-proxy shared-memory accesses before later
// async-proxy (TMA) writes to the same buffer.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bulk copy `bytes` (multiple of 16, both addresses 16-byte aligned).
__device__ __forceinline__ void tma_bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// ---------------------------------------------------------------------------
// EUC_2D: nint(sqrt(dx^2+dy^2)) exactly.  sqrt(s) is never an exact
// half-integer for integer s, and the nearest integer r >= 1 to sqrt(s) is the
// one with (r - 1/2)^2 < s < (r + 1/2)^2, i.e. -r < s - r^2 <= r.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Small coordinates: s < 2^24 (checked on the host), fp32 path.  The nearest
// integer to the approximate root is off by at most one; one step either way
// by the test above makes it exact (s = 0 steps to -1 and is clamped).
__device__ __forceinline__ int euc2d_small(int ax, int ay, int bx, int by) {
    const int dx = ax - bx, dy = ay - by;
    const int s = dx * dx + dy * dy;
    int r = __float2int_rn(sqrt_approx(static_cast<float>(s)));
    const int e = s - r * r;
    r += (e > r) ? 1 : ((e <= -r) ? -1 : 0);
    return max(r, 0);
}

// General coordinates (|coord| <= 2^20): int64 square, fp64 estimate.
__device__ __forceinline__ int euc2d_exact(long long ax, long long ay, long long bx, long long by) {
    long long dx = ax - bx, dy = ay - by;
    long long s = dx * dx + dy * dy;
    long long r = static_cast<long long>(sqrt(static_cast<double>(s)));
    while (r * r > s) --r;
    while ((r + 1) * (r + 1) <= s) ++r;
    return static_cast<int>(r + ((s - r * r) > r ? 1 : 0));
}

// ---------------------------------------------------------------------------
// Counter-based RNG: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014).  The
// draw for (key, counter) is the (counter+1)-th output of the generator
// seeded with key: the state key + (counter+1)*gamma through the finaliser.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t sm64_finalise(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t draw(uint64_t key, uint64_t counter) {
    return sm64_finalise(key + (counter + 1ull) * 0x9E3779B97F4A7C15ull);
}
enum : uint64_t { RNG_STREAM_ALNS = 1, RNG_STREAM_BRKGA = 2, RNG_STREAM_WARM = 3 };
__host__ __device__ __forceinline__ uint64_t stream_key(uint64_t seed, uint64_t stream) {
    return draw(seed, stream);
}
// integer in [0, k): top 32 bits times k, high word
__host__ __device__ __forceinline__ int draw_below(uint64_t r, int k) {
    return static_cast<int>(((r >> 32) * static_cast<uint64_t>(k)) >> 32);
}
// double in [0,1) with 53 random bits (exact conversion and scaling)
__device__ __forceinline__ double draw_unit(uint64_t r) {
    return __dmul_rn(static_cast<double>(r >> 11), 1.0 / 9007199254740992.0);
}
// float key in [0,1) with 24 random bits (exact)
__device__ __forceinline__ float draw_key(uint64_t r) {
    return __fmul_rn(static_cast<float>(static_cast<uint32_t>(r >> 40)), 1.0f / 16777216.0f);
}

// ---------------------------------------------------------------------------
// exp for the simulated-annealing test.  Cody-Waite argument reduction
// x = k*ln2 + r (ln2 as a 32-bit-mantissa head plus a tail so k*head is
// exact), then the degree-20 Taylor polynomial of e^r in Horner form, then
// scaling by 2^k built from its exponent bits.  Every operation is an
// explicitly rounded intrinsic, so nothing is contracted into an FMA.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double exp_sa(double x) {
    if (x != x) return x;
    if (x > 709.0) return __longlong_as_double(0x7ff0000000000000ll);
    if (x < -708.0) return 0.0;
    const double ln2_hi = 0.693147180369123816490;
    const double ln2_lo = 1.90821492927058770002e-10;
    const double inv_ln2 = 1.44269504088896338700;
    double kd = floor(__dadd_rn(__dmul_rn(x, inv_ln2), 0.5));
    int k = static_cast<int>(kd);
    double r = __dsub_rn(__dsub_rn(x, __dmul_rn(kd, ln2_hi)), __dmul_rn(kd, ln2_lo));
    double s = 1.0;
    for (int j = 20; j >= 1; --j) s = __dadd_rn(1.0, __dmul_rn(s, __ddiv_rn(r, static_cast<double>(j))));
    double scale = __longlong_as_double(static_cast<long long>(k + 1023) << 52);
    return __dmul_rn(s, scale);
}

}  // namespace vrp
