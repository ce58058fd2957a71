// Host-side pieces shared by the library's translation units: the graph
// object behind the opaque ldpc_graph handle, its cached decode workspace,
// CUDA-to-status mapping and a guard that restores the caller's device.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/ldpc.h"
#include "device_types.h"

namespace ldpcgb {

struct Workspace {
    void* buf = nullptr;
    size_t cap = 0;
    Ctrl* ctrl = nullptr;      // separate small allocation
    int* host_err = nullptr;   // pinned
    unsigned long long* host_iters = nullptr;  // pinned
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    // staging for ldpc_decode_host
    void* stage = nullptr;
    size_t stage_cap = 0;
    // dependency lists of the dataflow schedule, for the codes and item sizes in deps_key
    void* deps = nullptr;
    std::vector<long long> deps_key;
    std::vector<size_t> deps_off;  // per code: cn_ptr, cn_dep, vn_ptr, vn_dep (int offsets into deps)
    // guard regions of the last decode that asked for them (debug_guards), byte offsets into buf
    std::vector<size_t> guard_off;
};

}  // namespace ldpcgb

struct ldpc_graph {
    int kind = 0;  // 0 = CSR, 1 = QC
    int device = 0;
    int32_t m = 0, n = 0;
    int64_t E = 0;
    // QC description
    int mb = 0, nb = 0, Z = 0, nblk = 0;
    // device arrays (one allocation)
    void* dmem = nullptr;
    ldpcgb::QcDev qc{};
    ldpcgb::CsrDev csr{};
    int vn_tiles = 0, cn_tiles = 0;
    std::vector<int> row_deg, col_deg;  // QC base-matrix row and column weights
    // host copies of the QC tables (as QcDev holds them on the device)
    std::vector<int> h_row_ptr, h_blk_col, h_blk_shift, h_col_ptr, h_col_blk, h_blk_row;
    ldpcgb::Workspace ws;
};

namespace ldpcgb {

inline ldpc_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return LDPC_OK;
    if (e == cudaErrorMemoryAllocation) return LDPC_ERR_OOM;
    return LDPC_ERR_CUDA;
}

#define LDPC_TRY(expr)                                   \
    do {                                                 \
        ldpc_status st_ = ldpcgb::cuda_status(expr);     \
        if (st_ != LDPC_OK) return st_;                  \
    } while (0)

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Graph, device class map (validated at plan creation), iterations and
// classes of a weighted-BP plan, for decoding with its learned weights.
bool wbp_plan_classes(const ldpc_wbp* plan, const ldpc_graph** graph, const int** cls, int* iters, int* classes);

// An NVTX range around one library call (visible in Nsight Systems / Compute;
// costs a few nanoseconds when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    cudaError_t enter(int dev) {
        cudaError_t e = cudaGetDevice(&prev);
        if (e != cudaSuccess) return e;
        if (prev != dev) {
            e = cudaSetDevice(dev);
            changed = e == cudaSuccess;
        }
        return e;
    }
    ~DeviceGuard() {
        if (changed) cudaSetDevice(prev);
    }
};

}  // namespace ldpcgb
