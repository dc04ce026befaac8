// Host-side internals shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/vrprpd.h"

namespace vrp {

void set_error(const char* fmt, ...);

// Raise a kernel's dynamic shared-memory limit to everything the device
// allows, once per (kernel, device).  The limit is per-function global state,
// so setting it per launch would race between host threads that launch the
// same kernel with different sizes; the size a launch uses is its own.
int ensure_smem_limit(const void* kernel);
// The three-phase start and its refinement by a team of team_blocks CTAs (0:
// chosen from n); the server passes each request's share (alns.cu).
int initial_solution_paper_tb(const vrprpd_instance* I, int32_t refine_rounds, vrprpd_solution* out,
                              cudaStream_t stream, int team_blocks);
// The paper's three-phase initial solution into device buffers (construct.cu).
int construct_paper_device(const vrprpd_instance* I, int32_t* ops, int32_t* off, cudaStream_t stream);

// Coordinates present and small enough (squared extent < 2^24) for the exact
// fp32 EUC_2D path of the kernels.
bool coords_exact_small(const vrprpd_instance* I);

#define VRP_CUDA(call)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            ::vrp::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),     \
                             __FILE__, __LINE__);                                        \
            return VRPRPD_ECUDA;                                                         \
        }                                                                                \
    } while (0)

#define VRP_CHECK(cond, code, ...)        \
    do {                                  \
        if (!(cond)) {                    \
            ::vrp::set_error(__VA_ARGS__); \
            return (code);                \
        }                                 \
    } while (0)

// Device-side error words (written by kernels, read by vrprpd_sync).
enum : int { DEV_OK = 0, DEV_TIMEOUT_TMA = 1, DEV_TIMEOUT_BARRIER = 2, DEV_BAD_STATE = 3 };

struct EvalTuning {
    int dist_mode = VRPRPD_DIST_AUTO;
    int warps_per_block = 0;
    int blocks_per_sm = 0;
    int walk = VRPRPD_WALK_STAGED;
    int group_warps = 1;
};

}  // namespace vrp

struct vrprpd_instance {
    int32_t n = 0, m = 0, R = 0, Q = 0;
    uint32_t flags = 0;
    int device = 0;
    int num_sms = 0;
    size_t smem_optin = 0;
    int32_t maxd = 0, maxp = 0;
    bool has_coords = false;
    bool has_d16 = false;
    // device arrays (library-owned, 256-byte aligned, sizes padded to 16 bytes)
    int32_t* d32 = nullptr;      // (n+1)^2
    uint16_t* d16 = nullptr;     // (n+1)^2 when maxd < 65536
    int32_t* coords = nullptr;   // (n+1) x 2
    int32_t* p = nullptr;        // n+1, p[0] = 0, p[c] = processing time of c
    int* err = nullptr;          // device error word
    // host copies
    std::vector<int32_t> h_d, h_p, h_coords;
    // plain-form scratch, grown on demand
    int32_t* plain_scratch = nullptr;
    size_t plain_scratch_words = 0;
    // host staging for vrprpd_evaluate_host
    int32_t* stage = nullptr;
    size_t stage_bytes = 0;
    vrp::EvalTuning tune;
    vrp::EvalTuning tune_staged;   // the best staged-walk shape the autotuner saw (host-mapped candidates)
};
