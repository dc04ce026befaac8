// Instance construction: validation, device residency and the EUC_2D
// distance kernel (Section 5.1: TSPLIB edge weights as travel times).
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <set>
#include <utility>

#include "device_common.cuh"
#include "internal.h"

namespace vrp {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

// d(i,j) for all pairs; one thread per entry; also tracks max(d).
__global__ void euc2d_kernel(const int32_t* __restrict__ coords, int N, int32_t* __restrict__ d32,
                             int* __restrict__ maxd) {
    long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    long long total = static_cast<long long>(N) * N;
    int local_max = 0;
    for (; idx < total; idx += static_cast<long long>(gridDim.x) * blockDim.x) {
        int i = static_cast<int>(idx / N), j = static_cast<int>(idx - static_cast<long long>(i) * N);
        int v = euc2d_exact(coords[2 * i], coords[2 * i + 1], coords[2 * j], coords[2 * j + 1]);
        d32[idx] = v;
        local_max = v > local_max ? v : local_max;
    }
    for (int o = 16; o > 0; o >>= 1) local_max = max(local_max, __shfl_xor_sync(FULL_MASK, local_max, o));
    if ((threadIdx.x & 31) == 0) atomicMax(maxd, local_max);
}

__global__ void narrow16_kernel(const int32_t* __restrict__ d32, uint16_t* __restrict__ d16, long long total) {
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        d16[i] = static_cast<uint16_t>(d32[i]);
}

int ensure_smem_limit(const void* kernel) {
    static std::mutex mu;
    static std::set<std::pair<const void*, int>> done;
    int dev = 0;
    VRP_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({kernel, dev})) return VRPRPD_OK;
    cudaFuncAttributes fa{};
    VRP_CUDA(cudaFuncGetAttributes(&fa, kernel));
    int optin = 0;
    VRP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    VRP_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  optin - static_cast<int>(fa.sharedSizeBytes)));
    done.insert({kernel, dev});
    return VRPRPD_OK;
}

static size_t pad16(size_t bytes) { return (bytes + 15) & ~static_cast<size_t>(15); }

static int finish_create(vrprpd_instance* I, vrprpd_instance** out) {
    const int N = I->n + 1;
    const long long NN = static_cast<long long>(N) * N;
    // schedule-time bound: a path enters each op by a route edge or a pickup
    // edge once and ends with a return leg
    long long bound = (2ll * I->n + 1) * I->maxd + static_cast<long long>(I->n) * I->maxp;
    if (bound > 2147483646ll) {
        set_error("instance too large for int32 schedule times: (2n+1)*max(d) + n*max(p) = %lld", bound);
        return VRPRPD_EINVAL;
    }
    if (I->maxd < 65536) {
        VRP_CUDA(cudaMalloc(&I->d16, pad16(NN * sizeof(uint16_t))));
        narrow16_kernel<<<256, 256>>>(I->d32, I->d16, NN);
        VRP_CUDA(cudaGetLastError());
        I->has_d16 = true;
    }
    VRP_CUDA(cudaMalloc(&I->err, 16));
    VRP_CUDA(cudaMemset(I->err, 0, 16));
    VRP_CUDA(cudaStreamSynchronize(nullptr));   // this creation's own work only
    *out = I;
    return VRPRPD_OK;
}

static int common_init(vrprpd_instance* I, const int32_t* p, int32_t n, int32_t m, int32_t R, int32_t Q,
                       uint32_t flags) {
    VRP_CHECK(n >= 1 && n <= (1 << 20), VRPRPD_EINVAL, "n=%d out of range [1, 2^20]", n);
    VRP_CHECK(m >= 1 && m <= 4096, VRPRPD_EINVAL, "m=%d out of range [1, 4096]", m);
    VRP_CHECK(R >= 0 && Q >= 1, VRPRPD_EINVAL, "need R >= 0 and Q >= 1 (R=%d Q=%d)", R, Q);
    VRP_CHECK(flags == VRPRPD_LOAD_MIN || flags == VRPRPD_LOAD_FULL, VRPRPD_EINVAL, "bad flags %u", flags);
    VRP_CHECK(p != nullptr, VRPRPD_EINVAL, "p is NULL");
    I->n = n;
    I->m = m;
    I->R = R;
    I->Q = Q;
    I->flags = flags;
    I->h_p.assign(n + 1, 0);
    for (int c = 1; c <= n; ++c) {
        VRP_CHECK(p[c - 1] >= 0, VRPRPD_EINVAL, "p[%d] = %d is negative", c - 1, p[c - 1]);
        I->h_p[c] = p[c - 1];
        I->maxp = I->h_p[c] > I->maxp ? I->h_p[c] : I->maxp;
    }
    VRP_CUDA(cudaGetDevice(&I->device));
    VRP_CUDA(cudaDeviceGetAttribute(&I->num_sms, cudaDevAttrMultiProcessorCount, I->device));
    int optin = 0;
    VRP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, I->device));
    I->smem_optin = static_cast<size_t>(optin);
    VRP_CUDA(cudaMalloc(&I->p, pad16((n + 1) * sizeof(int32_t))));
    VRP_CUDA(cudaMemcpy(I->p, I->h_p.data(), (n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
    return VRPRPD_OK;
}

}  // namespace vrp

using namespace vrp;

extern "C" int vrprpd_instance_create(const int32_t* coords, const int32_t* p, int32_t n, int32_t m,
                                      int32_t R, int32_t Q, uint32_t flags, vrprpd_instance** out) {
    VRP_CHECK(out != nullptr && coords != nullptr, VRPRPD_EINVAL, "coords/out is NULL");
    *out = nullptr;
    vrprpd_instance* I = new vrprpd_instance();
    int rc = common_init(I, p, n, m, R, Q, flags);
    if (rc != VRPRPD_OK) { vrprpd_instance_destroy(I); return rc; }
    const int N = n + 1;
    for (int i = 0; i < 2 * N; ++i)
        if (coords[i] > (1 << 20) || coords[i] < -(1 << 20)) {
            set_error("coordinate %d out of range [-2^20, 2^20]", coords[i]);
            vrprpd_instance_destroy(I);
            return VRPRPD_EINVAL;
        }
    I->h_coords.assign(coords, coords + 2 * N);
    I->has_coords = true;
    const long long NN = static_cast<long long>(N) * N;
    int* dmax = nullptr;
    cudaError_t e = cudaMalloc(&I->coords, pad16(2 * N * sizeof(int32_t)));
    if (e == cudaSuccess) e = cudaMalloc(&I->d32, pad16(NN * sizeof(int32_t)));
    if (e == cudaSuccess) e = cudaMalloc(&dmax, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(I->coords, coords, 2 * N * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(dmax, 0, sizeof(int));
    if (e == cudaSuccess) {
        int blocks = static_cast<int>((NN + 255) / 256);
        blocks = blocks > 4096 ? 4096 : blocks;
        euc2d_kernel<<<blocks, 256>>>(I->coords, N, I->d32, dmax);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&I->maxd, dmax, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) {
        I->h_d.resize(NN);
        e = cudaMemcpy(I->h_d.data(), I->d32, NN * sizeof(int32_t), cudaMemcpyDeviceToHost);
    }
    if (dmax) cudaFree(dmax);
    if (e != cudaSuccess) {
        set_error("instance_create: %s", cudaGetErrorString(e));
        vrprpd_instance_destroy(I);
        return VRPRPD_ECUDA;
    }
    rc = finish_create(I, out);
    if (rc != VRPRPD_OK) vrprpd_instance_destroy(I);
    return rc;
}

extern "C" int vrprpd_instance_create_dist(const int32_t* d, const int32_t* p, int32_t n, int32_t m,
                                           int32_t R, int32_t Q, uint32_t flags, vrprpd_instance** out) {
    VRP_CHECK(out != nullptr && d != nullptr, VRPRPD_EINVAL, "d/out is NULL");
    *out = nullptr;
    vrprpd_instance* I = new vrprpd_instance();
    int rc = common_init(I, p, n, m, R, Q, flags);
    if (rc != VRPRPD_OK) { vrprpd_instance_destroy(I); return rc; }
    const long long NN = static_cast<long long>(n + 1) * (n + 1);
    for (long long i = 0; i < NN; ++i) {
        if (d[i] < 0) {
            set_error("d[%lld] = %d is negative", i, d[i]);
            vrprpd_instance_destroy(I);
            return VRPRPD_EINVAL;
        }
        I->maxd = d[i] > I->maxd ? d[i] : I->maxd;
    }
    I->h_d.assign(d, d + NN);
    cudaError_t e = cudaMalloc(&I->d32, pad16(NN * sizeof(int32_t)));
    if (e == cudaSuccess) e = cudaMemcpy(I->d32, d, NN * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        set_error("instance_create_dist: %s", cudaGetErrorString(e));
        vrprpd_instance_destroy(I);
        return VRPRPD_ECUDA;
    }
    rc = finish_create(I, out);
    if (rc != VRPRPD_OK) vrprpd_instance_destroy(I);
    return rc;
}

extern "C" void vrprpd_instance_destroy(vrprpd_instance* I) {
    if (!I) return;
    cudaFree(I->d32);
    cudaFree(I->d16);
    cudaFree(I->coords);
    cudaFree(I->p);
    cudaFree(I->err);
    cudaFree(I->plain_scratch);
    cudaFree(I->stage);
    delete I;
}

extern "C" int vrprpd_instance_get_dist(const vrprpd_instance* I, int32_t* d_host) {
    VRP_CHECK(I && d_host, VRPRPD_EINVAL, "NULL argument");
    std::memcpy(d_host, I->h_d.data(), I->h_d.size() * sizeof(int32_t));
    return VRPRPD_OK;
}

extern "C" int vrprpd_sync(const vrprpd_instance* I, void* stream) {
    VRP_CHECK(I, VRPRPD_EINVAL, "NULL instance");
    VRP_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    int err = 0;
    VRP_CUDA(cudaMemcpy(&err, I->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err != DEV_OK) {
        VRP_CUDA(cudaMemset(I->err, 0, sizeof(int)));
        set_error("device-side error %d (bounded wait gave up)", err);
        return VRPRPD_ETIMEOUT;
    }
    return VRPRPD_OK;
}

extern "C" const char* vrprpd_last_error(void) { return g_err; }
