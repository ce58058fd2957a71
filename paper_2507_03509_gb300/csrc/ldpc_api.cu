// C ABI of the GB300 syndrome-based sum-product LDPC decoder (include/ldpc.h).
//
// Host side: validates graphs and arguments, keeps a device copy of each
// graph and a workspace that grows on demand, packs the syndrome, launches
// the cooperative persistent decoder (bp_kernels.cuh) and reads back one
// status word.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include "../../include/ldpc.h"
#include "bp_kernels.cuh"
#include "flow_kernel.cuh"
#include "frame_kernel.cuh"
#include "host_common.h"

using namespace ldpcgb;

namespace {

constexpr unsigned long long kBarrierTimeoutNs = 10ull * 1000ull * 1000ull * 1000ull;  // 10 s
constexpr double kStepBytes = 192e6;  // default algorithmic bytes per group step (frames in flight)

// Upload a set of host int arrays into one device allocation.
ldpc_status upload_arrays(const std::vector<std::vector<int>>& arrays, void** dmem,
                          std::vector<const int*>& dptrs) {
    size_t total = 0;
    std::vector<size_t> off;
    for (const auto& a : arrays) {
        off.push_back(total);
        total += ((a.size() * sizeof(int) + 255) / 256) * 256;
    }
    if (total == 0) total = 256;
    void* d = nullptr;
    LDPC_TRY(cudaMalloc(&d, total));
    for (size_t i = 0; i < arrays.size(); ++i) {
        if (!arrays[i].empty()) {
            cudaError_t e = cudaMemcpy((char*)d + off[i], arrays[i].data(), arrays[i].size() * sizeof(int),
                                       cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                cudaFree(d);
                return cuda_status(e);
            }
        }
        dptrs.push_back((const int*)((char*)d + off[i]));
    }
    *dmem = d;
    return LDPC_OK;
}

void free_workspace(Workspace& ws) {
    if (ws.buf) cudaFree(ws.buf);
    if (ws.ctrl) cudaFree(ws.ctrl);
    if (ws.host_err) cudaFreeHost(ws.host_err);
    if (ws.host_iters) cudaFreeHost(ws.host_iters);
    if (ws.stage) cudaFree(ws.stage);
    if (ws.deps) cudaFree(ws.deps);
    for (auto& e : ws.ev)
        if (e) cudaEventDestroy(e);
    ws = Workspace{};
}

// Device layout of one decode's state.
struct Layout {
    size_t c2v, app, qpart, q0part, qval, q0val, unsat, sbits, new_frame, total;
    std::vector<size_t> guards;  // offsets of the guard regions (debug_guards), kGuardBytes each
};

constexpr size_t kGuardBytes = 256;          // guard region before and after every array (debug_guards)
constexpr unsigned char kGuardByte = 0xA5;   // its fill byte

// Carves consecutive 256-byte aligned regions; with guards, a guard region
// precedes every region and one follows the last.
struct Carver {
    size_t off = 0;
    bool guard = false;
    std::vector<size_t>* guards = nullptr;
    size_t take(size_t bytes) {
        if (guard) {
            guards->push_back(off);
            off += kGuardBytes;
        }
        const size_t at = off;
        off = align_up(off + bytes, 256);
        return at;
    }
    size_t end() {
        if (guard) {
            guards->push_back(off);
            off += kGuardBytes;
        }
        return off;
    }
};

Layout make_layout(int slots, size_t elem, long long slot_E, int slot_n, int slot_nqb, long long sbits_words,
                   bool guard) {
    Layout L{};
    Carver cv;
    cv.guard = guard;
    cv.guards = &L.guards;
    L.c2v = cv.take((size_t)slots * (size_t)slot_E * elem);
    L.app = cv.take((size_t)slots * (size_t)slot_n * elem);
    L.qpart = cv.take((size_t)slots * slot_nqb * kWarps * sizeof(double));
    L.q0part = cv.take((size_t)slots * slot_nqb * kWarps * sizeof(double));
    L.qval = cv.take((size_t)slots * kQParts * sizeof(double));
    L.q0val = cv.take((size_t)slots * kQParts * sizeof(double));
    L.unsat = cv.take(2 * (size_t)slots * sizeof(int));
    L.sbits = cv.take((size_t)sbits_words * sizeof(unsigned));
    L.new_frame = cv.take((size_t)slots * sizeof(int));
    L.total = cv.off;  // the dataflow schedule carves on from here; end() closes the last guard
    return L;
}

// Fill the guard regions of this launch's layout (debug_guards) and remember
// them for ldpc_*_check_guards.
ldpc_status fill_guards(Workspace& ws, const std::vector<size_t>& guards, cudaStream_t stream) {
    ws.guard_off = guards;
    for (size_t off : guards)
        LDPC_TRY(cudaMemsetAsync((char*)ws.buf + off, kGuardByte, kGuardBytes, stream));
    return LDPC_OK;
}

// Whether every guard region of the last guarded launch still holds its fill.
ldpc_status check_guards(Workspace& ws, int device) {
    if (ws.guard_off.empty() || !ws.buf) return LDPC_ERR_INVALID_ARG;
    DeviceGuard guard;
    LDPC_TRY(guard.enter(device));
    LDPC_TRY(cudaDeviceSynchronize());
    std::vector<unsigned char> h(kGuardBytes);
    for (size_t off : ws.guard_off) {
        LDPC_TRY(cudaMemcpy(h.data(), (char*)ws.buf + off, kGuardBytes, cudaMemcpyDeviceToHost));
        for (unsigned char b : h)
            if (b != kGuardByte) return LDPC_ERR_BOUNDS;
    }
    return LDPC_OK;
}

ldpc_status ensure_workspace(Workspace& ws, size_t bytes) {
    if (!ws.ctrl) {
        LDPC_TRY(cudaMalloc(&ws.ctrl, kMaxGroups * sizeof(Ctrl)));
        LDPC_TRY(cudaHostAlloc(&ws.host_err, sizeof(int), cudaHostAllocDefault));
        LDPC_TRY(cudaHostAlloc(&ws.host_iters, sizeof(unsigned long long), cudaHostAllocDefault));
        for (auto& e : ws.ev) LDPC_TRY(cudaEventCreate(&e));
    }
    if (ws.cap < bytes) {
        if (ws.buf) {
            cudaFree(ws.buf);
            ws.buf = nullptr;
            ws.cap = 0;
        }
        LDPC_TRY(cudaMalloc(&ws.buf, bytes));
        ws.cap = bytes;
    }
    return LDPC_OK;
}

const QcDev& code_of(const ldpc_graph* g, QcDev*) { return g->qc; }
const CsrDev& code_of(const ldpc_graph* g, CsrDev*) { return g->csr; }

// One decode launch: frames of 1..kMaxCodes codes (graphs of one kind), with
// optional per-frame device arrays (code index, offsets into the concatenated
// buffers; NULL = one code, frames back to back).
struct Job {
    const ldpc_graph* const* graphs;
    int ngraphs;
    int frames;
    const int* frame_code;       // device [frames] or NULL
    const long long* var_off;    // device [frames] or NULL
    const long long* syn_off;    // device [frames] or NULL (syndrome bytes)
    const long long* sb_off;     // device [frames] or NULL (packed words)
    long long sbits_words;       // packed syndrome words of all frames
    int max_slot_frames;         // frames that may run at once (min(frames, ...))
    const float* llr;
    const uint8_t* syndrome;
    uint8_t* bits_out;
    uint8_t* flags_out;
    int32_t* iters_out;
    int max_iter, rule;
    bool var_unaligned[kMaxCodes];  // some frame of code c starts at an offset not a multiple of 4
    const float* wts;            // learned weights [w_iters][w_classes] or NULL
    const int* wcls;             // class of each base block (QC) / edge (CSR)
    int w_iters, w_classes;
    int cn_chunk[kMaxCodes];     // QC item sizes chosen by a caller (0: the model's pick)
    int vn_chunk[kMaxCodes];
};

// QC item sizes: simulate the static assignment (item it goes to CTA it mod
// gsize) of one step of the group's slots and take the size whose busiest CTA
// has the least work (checks or variables times (degree + 1), plus a fixed
// cost per item).
void pick_chunks(const ldpc_graph* g, int gsize, int slots_per_group, int* cn_chunk, int* cn_tiles, int* vn_chunk,
                 int* vn_tiles) {
    std::vector<long long> load((size_t)gsize);
    auto pick = [&](const std::vector<int>& deg, const int* cand, int ncand, int* chunk, int* tiles) {
        long long best = -1;
        for (int c = 0; c < ncand; ++c) {
            const int per = (g->Z + cand[c] - 1) / cand[c];
            std::fill(load.begin(), load.end(), 0LL);
            long long it = 0;
            for (int sl = 0; sl < slots_per_group; ++sl)
                for (int r = 0; r < (int)deg.size(); ++r)
                    for (int q = 0; q < per; ++q, ++it) {
                        const int len = std::min(cand[c], g->Z - q * cand[c]);
                        load[(size_t)(it % gsize)] += (long long)len * (deg[r] + 1) + 2048;
                    }
            const long long worst = *std::max_element(load.begin(), load.end());
            if (best < 0 || worst < best) {
                best = worst;
                *chunk = cand[c];
                *tiles = (int)deg.size() * per;
            }
        }
    };
    static const int cn_cand[] = {512, 1024, 2048, 4096};
    static const int vn_cand[] = {1024, 2048, 4096, 8192};
    pick(g->row_deg, cn_cand, 4, cn_chunk, cn_tiles);
    pick(g->col_deg, vn_cand, 4, vn_chunk, vn_tiles);
}

// Largest sizes over a job's codes: slots are sized for the largest code.
struct SlotSizes {
    long long E;
    int n, nqb, cn_max, vn_max;
};

// Per-code sizes of a job (item sizes from the model for a group of gsize CTAs
// and slots_per_group slots, unless the job fixes them) and the pack table.
template <class Code>
void code_set(const Job& job, int gsize, int slots_per_group, CodeSet<Code>& cs, SlotSizes& sz, PackInfo& pi) {
    cs.count = job.ngraphs;
    long long slot_E = 0;
    int slot_n = 0, slot_nqb = 0, cn_max = 0, vn_max = 0;
    for (int c = 0; c < job.ngraphs; ++c) {
        const ldpc_graph* g = job.graphs[c];
        CodeInfo<Code>& ci = cs.c[c];
        ci.code = code_of(g, (Code*)nullptr);
        ci.n = g->n;
        ci.m = g->m;
        ci.E = g->E;
        ci.swords = (g->m + 31) / 32;
        ci.cn_tiles = g->cn_tiles;
        ci.vn_tiles = g->vn_tiles;
        ci.cn_chunk = kQcCnChunk;
        ci.vn_chunk = kQcVnChunk;
        ci.nqb = g->vn_tiles;
        ci.vec4 = 0;
        if (g->kind == 1) {
            pick_chunks(g, gsize, slots_per_group, &ci.cn_chunk, &ci.cn_tiles, &ci.vn_chunk, &ci.vn_tiles);
            if (job.cn_chunk[c] > 0) {  // measured by the batch autotuner
                ci.cn_chunk = job.cn_chunk[c];
                ci.cn_tiles = g->mb * ((g->Z + ci.cn_chunk - 1) / ci.cn_chunk);
            }
            if (job.vn_chunk[c] > 0) {
                ci.vn_chunk = job.vn_chunk[c];
                ci.vn_tiles = g->nb * ((g->Z + ci.vn_chunk - 1) / ci.vn_chunk);
            }
            ci.nqb = g->nb * ((g->Z + kQBlock - 1) / kQBlock);
            // 16-byte variable-side loads: Z % 4 == 0 and every frame's Lch and
            // decisions 16-byte aligned (the buffer aligned, every frame of the
            // code at an offset that is a multiple of 4)
            ci.vec4 = ((g->Z % 4) == 0 && ((uintptr_t)job.llr % 16) == 0 && !job.var_unaligned[c]) ? 1 : 0;
        }
        // slot strides rounded up to 64 elements, so every slot's messages and
        // APP values start 256-byte aligned whatever the codes' sizes
        slot_E = std::max(slot_E, (long long)align_up((size_t)ci.E, 64));
        slot_n = std::max(slot_n, (int)align_up((size_t)ci.n, 64));
        slot_nqb = std::max(slot_nqb, ci.nqb);
        cn_max = std::max(cn_max, ci.cn_tiles);
        vn_max = std::max(vn_max, ci.vn_tiles);
        pi.m[c] = ci.m;
        pi.swords[c] = ci.swords;
    }
    pi.frame_code = job.frame_code;
    pi.syn_off = job.syn_off;
    pi.sb_off = job.sb_off;
    sz.E = slot_E;
    sz.n = slot_n;
    sz.nqb = slot_nqb;
    sz.cn_max = cn_max;
    sz.vn_max = vn_max;
}

// The end of every decode launch.  Asynchronous (status_out set): the device
// status word is written by a kernel, nothing waits.  Synchronous: the error
// word and the iteration total are read back, stats filled from the events
// ev[0] (start), ev[1]/ev[2] (around the persistent kernel) and ev[3] (end).
ldpc_status finish_decode(Workspace& ws, const ldpc_decode_opts& o, cudaStream_t stream, int32_t* status_out,
                          int grid, int slots) {
    const bool timing = o.stats != nullptr && status_out == nullptr;
    if (status_out) {
        status_kernel<<<1, 1, 0, stream>>>(ws.ctrl, status_out);
        LDPC_TRY(cudaGetLastError());
        return LDPC_OK;
    }
    LDPC_TRY(cudaMemcpyAsync(ws.host_err, &ws.ctrl->err, sizeof(int), cudaMemcpyDeviceToHost, stream));
    LDPC_TRY(cudaMemcpyAsync(ws.host_iters, &ws.ctrl->frame_iters, sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost, stream));
    if (timing) LDPC_TRY(cudaEventRecord(ws.ev[3], stream));
    LDPC_TRY(cudaStreamSynchronize(stream));
    const int err = *ws.host_err;
    if (timing) {
        ldpc_decode_stats* sst = o.stats;
        cudaEventElapsedTime(&sst->kernel_ms, ws.ev[1], ws.ev[2]);
        cudaEventElapsedTime(&sst->total_ms, ws.ev[0], ws.ev[3]);
        sst->kernel_launches = 3;
        sst->grid_ctas = grid;
        sst->threads_per_cta = kThreads;
        sst->active_frames = slots;
        sst->frame_iterations = (int64_t)*ws.host_iters;
    }
    if (err == kErrSyndrome) return LDPC_ERR_INVALID_ARG;
    if (err == kErrTimeout) return LDPC_ERR_TIMEOUT;
    if (err == kErrBounds) return LDPC_ERR_BOUNDS;
    if (err != kErrNone) return LDPC_ERR_CUDA;
    return LDPC_OK;
}

// ---------------------------------------------------------------------------
// Dataflow schedule (flow_kernel.cuh): dependency lists and launcher.
// ---------------------------------------------------------------------------

// Items of the other pass that each item of a QC code waits for.  A check item
// (row i, checks [t0, t1)) reads APP at (t + shift_b) mod Z of each block b's
// column: the variable items of those columns covering that (wrapping) range.
// A variable item (column j, variables [u0, u1)) reads the messages of each
// block b of the column at offsets u, written by the check items of the block's
// row covering (u - shift_b) mod Z.
void flow_deps(const ldpc_graph* g, int cn_chunk, int vn_chunk, std::vector<int>& cn_ptr, std::vector<int>& cn_dep,
               std::vector<int>& vn_ptr, std::vector<int>& vn_dep) {
    const int Z = g->Z, mb = g->mb, nb = g->nb;
    const int per_row = (Z + cn_chunk - 1) / cn_chunk, per_col = (Z + vn_chunk - 1) / vn_chunk;
    const std::vector<int>&rp = g->h_row_ptr, &bc = g->h_blk_col, &bs = g->h_blk_shift, &cp = g->h_col_ptr,
                      &cbk = g->h_col_blk, &br = g->h_blk_row;
    // tiles of `chunk` covering the cyclic range [a, a + len) mod Z, offset by base
    auto cover = [&](int a, int len, int chunk, int base, std::vector<int>& out) {
        const int end = a + len;
        auto add = [&](int lo, int hi) {  // [lo, hi), 0 <= lo < hi <= Z
            for (int q = lo / chunk; q <= (hi - 1) / chunk; ++q) out.push_back(base + q);
        };
        if (end <= Z) {
            add(a, end);
        } else {
            add(a, Z);
            add(0, end - Z);
        }
    };
    cn_ptr.assign(1, 0);
    cn_dep.clear();
    for (int i = 0; i < mb; ++i)
        for (int q = 0; q < per_row; ++q) {
            const int t0 = q * cn_chunk, len = std::min(cn_chunk, Z - t0);
            std::vector<int> d;
            for (int b = rp[i]; b < rp[i + 1]; ++b) cover((t0 + bs[b]) % Z, len, vn_chunk, bc[b] * per_col, d);
            std::sort(d.begin(), d.end());
            d.erase(std::unique(d.begin(), d.end()), d.end());
            cn_dep.insert(cn_dep.end(), d.begin(), d.end());
            cn_ptr.push_back((int)cn_dep.size());
        }
    vn_ptr.assign(1, 0);
    vn_dep.clear();
    for (int j = 0; j < nb; ++j)
        for (int q = 0; q < per_col; ++q) {
            const int u0 = q * vn_chunk, len = std::min(vn_chunk, Z - u0);
            std::vector<int> d;
            for (int x = cp[j]; x < cp[j + 1]; ++x) {
                const int b = cbk[x];
                cover(((u0 - bs[b]) % Z + Z) % Z, len, cn_chunk, br[b] * per_row, d);
            }
            std::sort(d.begin(), d.end());
            d.erase(std::unique(d.begin(), d.end()), d.end());
            vn_dep.insert(vn_dep.end(), d.begin(), d.end());
            vn_ptr.push_back((int)vn_dep.size());
        }
}

// Device lists of every code of the job for its item sizes, cached in the
// workspace (rebuilt only when the codes or sizes change; not while capturing).
ldpc_status flow_upload_deps(Workspace& ws, const Job& job, const CodeSet<QcDev>& cs, bool capturing,
                             FlowParams& fp) {
    std::vector<long long> key;
    for (int c = 0; c < job.ngraphs; ++c) {
        key.push_back((long long)(intptr_t)job.graphs[c]);
        key.push_back(cs.c[c].cn_chunk);
        key.push_back(cs.c[c].vn_chunk);
    }
    if (ws.deps_key != key || !ws.deps) {
        if (capturing) return LDPC_ERR_INVALID_ARG;  // run one decode of this configuration before capturing
        std::vector<int> all;
        std::vector<size_t> off;
        for (int c = 0; c < job.ngraphs; ++c) {
            std::vector<int> a, b, d, e;
            flow_deps(job.graphs[c], cs.c[c].cn_chunk, cs.c[c].vn_chunk, a, b, d, e);
            for (const std::vector<int>* v : {&a, &b, &d, &e}) {
                off.push_back(all.size());
                all.insert(all.end(), v->begin(), v->end());
                all.resize(align_up(all.size(), 64), 0);
            }
        }
        if (ws.deps) cudaFree(ws.deps);
        ws.deps = nullptr;
        ws.deps_key.clear();
        LDPC_TRY(cudaMalloc(&ws.deps, std::max<size_t>(all.size(), 1) * sizeof(int)));
        LDPC_TRY(cudaMemcpy(ws.deps, all.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice));
        ws.deps_key = key;
        ws.deps_off = off;
    }
    const int* d = (const int*)ws.deps;
    for (int c = 0; c < job.ngraphs; ++c) {
        fp.dep[c].cn_ptr = d + ws.deps_off[4 * c];
        fp.dep[c].cn_dep = d + ws.deps_off[4 * c + 1];
        fp.dep[c].vn_ptr = d + ws.deps_off[4 * c + 2];
        fp.dep[c].vn_dep = d + ws.deps_off[4 * c + 3];
    }
    return LDPC_OK;
}

// One decode with the dataflow schedule (QC codes): one group over the whole
// grid, every frame in flight up to max_active_frames, the lag from the options.
template <typename T>
ldpc_status launch_flow(Workspace& ws, const Job& job, const ldpc_decode_opts& o, cudaStream_t stream,
                        int32_t* status_out) {
    const int frames = job.frames;
    auto kernel = job.wts ? bp_flow_kernel<T, true> : bp_flow_kernel<T, false>;
    int dev = 0, sms = 0, per_sm = 0, coop = 0;
    LDPC_TRY(cudaGetDevice(&dev));
    LDPC_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    LDPC_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (!coop) return LDPC_ERR_CUDA;
    LDPC_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0));
    if (per_sm < 1) return LDPC_ERR_CUDA;
    int grid = std::min(per_sm * sms, kMaxGrid);
    if (o.grid_ctas > 0) grid = std::min(grid, o.grid_ctas);
    int slots = o.max_active_frames > 0 ? o.max_active_frames : frames;
    slots = std::max(1, std::min(std::min(slots, job.max_slot_frames), kMaxSlots));
    const int lag = std::max(1, std::min(o.flow_lag > 0 ? o.flow_lag : 2, slots));

    CodeSet<QcDev> cs{};
    SlotSizes sz{};
    PackInfo pi{};
    code_set(job, grid, slots, cs, sz, pi);

    cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
    LDPC_TRY(cudaStreamIsCapturing(stream, &capturing));
    const bool cap = capturing != cudaStreamCaptureStatusNone;
    FlowParams fp{};
    ldpc_status st = flow_upload_deps(ws, job, cs, cap, fp);
    if (st != LDPC_OK) return st;

    Layout L = make_layout(slots, sizeof(T), sz.E, sz.n, sz.nqb, job.sbits_words, o.debug_guards != 0);
    Carver cv;
    cv.off = L.total;
    cv.guard = o.debug_guards != 0;
    cv.guards = &L.guards;
    const size_t o_cnf = cv.take((size_t)slots * sz.cn_max * sizeof(int));
    const size_t o_vnf = cv.take((size_t)slots * sz.vn_max * sizeof(int));
    const size_t o_cnt = cv.take(2 * (size_t)slots * sizeof(unsigned));
    const size_t o_uns = cv.take(2 * (size_t)slots * sizeof(int));
    const size_t o_dec = cv.take((size_t)slots * sizeof(int));
    const size_t o_rec = cv.take((size_t)slots * sizeof(unsigned long long));
    const size_t o_prv = cv.take((size_t)slots * sizeof(int));
    const size_t o_qpv = cv.take((size_t)slots * sizeof(double));
    const size_t o_ret = cv.take(sizeof(int));
    const size_t o_prg = cv.take(sizeof(unsigned));
    const size_t off = cv.end();
    if (cap && (ws.cap < off || !ws.ctrl)) return LDPC_ERR_INVALID_ARG;  // run one decode of this size first
    st = ensure_workspace(ws, off);
    if (st != LDPC_OK) return st;
    char* base = (char*)ws.buf;
    ws.guard_off.clear();
    if (o.debug_guards) {
        st = fill_guards(ws, L.guards, stream);
        if (st != LDPC_OK) return st;
    }

    Params<T> p{};
    p.frames = frames;
    p.max_iter = job.max_iter;
    p.rule = job.rule;
    p.vnr_first_iter = o.vnr_first_iter;
    p.lmax = T(o.clamp);
    p.frame_code = job.frame_code;
    p.var_off = job.var_off;
    p.sb_off = job.sb_off;
    p.llr = job.llr;
    p.sbits = (const unsigned*)(base + L.sbits);
    p.bits_out = job.bits_out;
    p.flags_out = job.flags_out;
    p.iters_out = job.iters_out;
    p.slots = slots;
    p.slot_E = sz.E;
    p.slot_n = sz.n;
    p.slot_nqb = sz.nqb;
    p.cn_tiles_max = sz.cn_max;
    p.vn_tiles_max = sz.vn_max;
    p.c2v = (T*)(base + L.c2v);
    p.app = (T*)(base + L.app);
    p.qpart = (double*)(base + L.qpart);
    p.q0part = (double*)(base + L.q0part);
    p.qval = (double*)(base + L.qval);
    p.q0val = (double*)(base + L.q0val);
    p.unsat = (int*)(base + L.unsat);
    p.ctrl = ws.ctrl;
    p.trace_iters = o.trace_iters;
    p.trace_c2v = (T*)o.trace_c2v;
    p.trace_app = (T*)o.trace_app;
    p.trace_q = o.trace_q;
    p.timeout_ns = o.barrier_timeout_ms > 0 ? (unsigned long long)o.barrier_timeout_ms * 1000000ull
                                            : kBarrierTimeoutNs;
    p.bar_extra = o.test_unreachable_barrier ? 1u : 0u;
    p.groups = 1;
    p.slots_per_group = slots;
    p.new_frame = (int*)(base + L.new_frame);
    p.wts = job.wts;
    p.wcls = job.wcls;
    p.w_iters = job.w_iters;
    p.w_classes = job.w_classes;

    fp.lag = lag;
    fp.cn_items = sz.cn_max;
    fp.vn_items = sz.vn_max;
    fp.cn_flag = (int*)(base + o_cnf);
    fp.vn_flag = (int*)(base + o_vnf);
    fp.cn_count = (unsigned*)(base + o_cnt);
    fp.unsat = (int*)(base + o_uns);
    fp.dec = (int*)(base + o_dec);
    fp.rec = (unsigned long long*)(base + o_rec);
    fp.prev = (int*)(base + o_prv);
    fp.qprev = (double*)(base + o_qpv);
    fp.retired = (int*)(base + o_ret);
    fp.progress = (unsigned*)(base + o_prg);

    const bool timing = o.stats != nullptr && status_out == nullptr;
    if (timing) LDPC_TRY(cudaEventRecord(ws.ev[0], stream));
    {
        const long long words = (long long)slots * (sz.cn_max + sz.vn_max);
        const int blocks = (int)std::max(1LL, std::min(1024LL, (words + 255) / 256));
        flow_init_kernel<<<blocks, 256, 0, stream>>>(fp, slots, frames, ws.ctrl);
        LDPC_TRY(cudaGetLastError());
    }
    {
        int max_words = 1;
        for (int c = 0; c < job.ngraphs; ++c) max_words = std::max(max_words, pi.swords[c]);
        const dim3 pgrid((unsigned)std::min((max_words + 31) / 32, 4096), (unsigned)std::max(1, std::min(frames, 65535)));
        pack_syndrome_kernel<<<pgrid, 256, 0, stream>>>(job.syndrome, frames, pi, (unsigned*)(base + L.sbits),
                                                        ws.ctrl);
        LDPC_TRY(cudaGetLastError());
    }
    if (timing) LDPC_TRY(cudaEventRecord(ws.ev[1], stream));
    {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;  // all CTAs resident: the item waits need it
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        LDPC_TRY(cudaLaunchKernelEx(&cfg, kernel, p, cs, fp));
    }
    if (timing) LDPC_TRY(cudaEventRecord(ws.ev[2], stream));
    return finish_decode(ws, o, stream, status_out, grid, slots);
}

// Shared memory a frame-per-CTA decode of this job's code needs, or 0 if the
// schedule does not apply (one CSR code; FP32; 16-bit indices; frame and
// index lists within 220 KB).
constexpr size_t kFrameSmemMax = 220 * 1024;
size_t frame_schedule_smem(const Job& job, bool fp64) {
    if (job.ngraphs != 1 || fp64 || job.graphs[0]->kind != 0) return 0;
    const ldpc_graph* g = job.graphs[0];
    const size_t b = frame_smem_bytes(g->E, g->n, g->m, g->vn_tiles, (g->m + 31) / 32);
    return b <= kFrameSmemMax ? b : 0;
}

// Launch configuration of the frame-per-cluster kernel: pairs of CTAs.
cudaLaunchConfig_t pair_config(int grid, size_t smem, cudaStream_t stream, cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kFrameThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

// One decode with the frame-per-CTA schedule (frame_kernel.cuh): every CTA
// (pair: every cluster of two CTAs) takes whole frames from the queue and
// decodes each in shared memory.  pair: 0 = automatic (pairs when every frame
// gets its own pair at once, so that more SMs work), 1 = one CTA per frame,
// 2 = a pair per frame.
ldpc_status launch_frame(Workspace& ws, const Job& job, const ldpc_decode_opts& o, cudaStream_t stream,
                         int32_t* status_out, size_t smem, int pair) {
    const int frames = job.frames;
    auto kernel1 = job.wts ? csr_frame_kernel<true, 1> : csr_frame_kernel<false, 1>;
    auto kernel2 = job.wts ? csr_frame_kernel<true, 2> : csr_frame_kernel<false, 2>;
    int dev = 0, sms = 0, per_sm = 0, pairs_fit = 0;
    LDPC_TRY(cudaGetDevice(&dev));
    LDPC_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    LDPC_TRY(cudaFuncSetAttribute(kernel1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    LDPC_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel1, kFrameThreads, smem));
    if (per_sm < 1) return LDPC_ERR_CUDA;
    if (pair != 1) {
        cudaLaunchAttribute attr[1];
        const cudaLaunchConfig_t cfg = pair_config(2, smem, nullptr, attr);
        cudaError_t e = cudaFuncSetAttribute(kernel2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveClusters(&pairs_fit, (const void*)kernel2, &cfg);
        if (e != cudaSuccess) {
            if (pair == 2) LDPC_TRY(e);
            (void)cudaGetLastError();  // automatic selection falls back to one CTA per frame
            pairs_fit = 0;
        }
        if (pair == 2 && pairs_fit < 1) return LDPC_ERR_CUDA;
        if (pair == 0) pair = (pairs_fit >= 1 && frames <= pairs_fit) ? 2 : 1;
    }
    int grid = 0, units = 0;  // CTAs, and frames decoded at once
    if (pair == 2) {
        units = std::min(std::min(pairs_fit, kMaxGrid / 2), frames);
        if (o.grid_ctas > 0) units = std::min(units, std::max(1, o.grid_ctas / 2));
        grid = 2 * units;
    } else {
        grid = std::min(std::min(per_sm * sms, kMaxGrid), frames);
        if (o.grid_ctas > 0) grid = std::min(grid, o.grid_ctas);
        units = grid;
    }
    CodeSet<CsrDev> cs{};
    SlotSizes sz{};
    PackInfo pi{};
    code_set(job, grid, 1, cs, sz, pi);
    Layout L = make_layout(1, sizeof(float), sz.E, sz.n, sz.nqb, job.sbits_words, o.debug_guards != 0);
    if (o.debug_guards) {
        L.guards.push_back(L.total);
        L.total += kGuardBytes;
    }
    cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
    LDPC_TRY(cudaStreamIsCapturing(stream, &capturing));
    if (capturing != cudaStreamCaptureStatusNone && (ws.cap < L.total || !ws.ctrl)) return LDPC_ERR_INVALID_ARG;
    ldpc_status st = ensure_workspace(ws, L.total);
    if (st != LDPC_OK) return st;
    char* base = (char*)ws.buf;
    ws.guard_off.clear();
    if (o.debug_guards) {
        st = fill_guards(ws, L.guards, stream);
        if (st != LDPC_OK) return st;
    }
    Params<float> p{};
    p.frames = frames;
    p.max_iter = job.max_iter;
    p.rule = job.rule;
    p.vnr_first_iter = o.vnr_first_iter;
    p.lmax = o.clamp;
    p.frame_code = job.frame_code;
    p.var_off = job.var_off;
    p.sb_off = job.sb_off;
    p.llr = job.llr;
    p.sbits = (const unsigned*)(base + L.sbits);
    p.bits_out = job.bits_out;
    p.flags_out = job.flags_out;
    p.iters_out = job.iters_out;
    p.slots = 1;
    p.slot_E = sz.E;
    p.slot_n = sz.n;
    p.slot_nqb = sz.nqb;
    p.cn_tiles_max = sz.cn_max;
    p.vn_tiles_max = sz.vn_max;
    p.c2v = (float*)(base + L.c2v);
    p.app = (float*)(base + L.app);
    p.qpart = (double*)(base + L.qpart);
    p.q0part = (double*)(base + L.q0part);
    p.ctrl = ws.ctrl;
    p.trace_iters = o.trace_iters;
    p.trace_c2v = (float*)o.trace_c2v;
    p.trace_app = (float*)o.trace_app;
    p.trace_q = o.trace_q;
    p.groups = 1;
    p.slots_per_group = 1;
    p.wts = job.wts;
    p.wcls = job.wcls;
    p.w_iters = job.w_iters;
    p.w_classes = job.w_classes;
    const bool timing = o.stats != nullptr && status_out == nullptr;
    if (timing) LDPC_TRY(cudaEventRecord(ws.ev[0], stream));
    init_ctrl_kernel<<<1, 256, 0, stream>>>(ws.ctrl, 1, 0, (int*)(base + L.unsat), 2);  // queue from frame 0
    LDPC_TRY(cudaGetLastError());
    {
        const dim3 pgrid((unsigned)std::max(1, std::min((pi.swords[0] + 31) / 32, 4096)),
                         (unsigned)std::max(1, std::min(frames, 65535)));
        pack_syndrome_kernel<<<pgrid, 256, 0, stream>>>(job.syndrome, frames, pi, (unsigned*)(base + L.sbits),
                                                        ws.ctrl);
        LDPC_TRY(cudaGetLastError());
    }
    if (timing) LDPC_TRY(cudaEventRecord(ws.ev[1], stream));
    {
        const CodeInfo<CsrDev>& ci = cs.c[0];
        const FrameSmem fl = frame_smem_layout(ci.E, ci.n, ci.m, ci.nqb, ci.swords);
        if (pair == 2) {
            cudaLaunchAttribute attr[1];
            const cudaLaunchConfig_t cfg = pair_config(grid, smem, stream, attr);
            LDPC_TRY(cudaLaunchKernelEx(&cfg, kernel2, p, ci, fl));
        } else {
            kernel1<<<grid, kFrameThreads, smem, stream>>>(p, ci, fl);
        }
    }
    LDPC_TRY(cudaGetLastError());
    if (timing) LDPC_TRY(cudaEventRecord(ws.ev[2], stream));
    return finish_decode(ws, o, stream, status_out, grid, units);
}

// Schedule of a job: lock-step unless the caller asks for dataflow (QC only).
// Measured at n = 1e6 with 32 frames, the dataflow schedule ran at half the
// lock-step rate: its items wait on the per-frame decision, a join over every
// check item of the frame, once per iteration.
template <typename T, class Code>
bool use_flow(const ldpc_decode_opts& o) {
    return std::is_same<Code, QcDev>::value && o.schedule == LDPC_SCHEDULE_DATAFLOW;
}

// Synchronous (status_out == NULL): reads the status back and fills stats.
// Asynchronous: copies the device status word to status_out and returns at
// once; nothing in it waits for the host, so it can be captured in a graph
// (the workspace must already be large enough: no allocation while capturing).
template <typename T, class Code>
ldpc_status launch_decode(Workspace& ws, const Job& job, const ldpc_decode_opts& o, cudaStream_t stream,
                          int32_t* status_out = nullptr) {
    if constexpr (std::is_same<Code, QcDev>::value) {
        if (use_flow<T, Code>(o)) return launch_flow<T>(ws, job, o, stream, status_out);
    }
    if constexpr (std::is_same<Code, CsrDev>::value && std::is_same<T, float>::value) {
        // frame per CTA: asked for, or automatic for one small CSR code (unless the
        // unreachable-barrier test hook asks for a grid barrier, which it has none of)
        const size_t smem = frame_schedule_smem(job, false);
        const bool frame_sched = o.schedule == LDPC_SCHEDULE_FRAME || o.schedule == LDPC_SCHEDULE_FRAME_PAIR;
        if (frame_sched && smem == 0) return LDPC_ERR_INVALID_ARG;
        if (smem && (frame_sched || (o.schedule == LDPC_SCHEDULE_AUTO && o.test_unreachable_barrier == 0)))
            return launch_frame(ws, job, o, stream, status_out, smem,
                                o.schedule == LDPC_SCHEDULE_FRAME ? 1 : (o.schedule == LDPC_SCHEDULE_FRAME_PAIR ? 2 : 0));
    }
    if (o.schedule == LDPC_SCHEDULE_FRAME || o.schedule == LDPC_SCHEDULE_FRAME_PAIR) return LDPC_ERR_INVALID_ARG;
    const int frames = job.frames;
    // the weighted kernel is a separate instantiation: the unweighted one carries no weight code
    auto kernel = job.wts ? bp_decode_kernel<T, Code, true> : bp_decode_kernel<T, Code, false>;
    int dev = 0, sms = 0, per_sm = 0, coop = 0;
    LDPC_TRY(cudaGetDevice(&dev));
    LDPC_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    LDPC_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (!coop) return LDPC_ERR_CUDA;
    // occupancy with the largest slot table we may use
    LDPC_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)decode_smem_bytes(kMaxSlots)));
    LDPC_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads,
                                                           decode_smem_bytes(std::min(frames, kMaxSlots))));
    if (per_sm < 1) return LDPC_ERR_CUDA;
    int grid = std::min(per_sm * sms, kMaxGrid);
    if (o.grid_ctas > 0) grid = std::min(grid, o.grid_ctas);
    // groups and slots: by default two groups per resident CTA per SM (at most
    // one per frame).  Measured at n = 1e6 with 32 frames, all in flight: 8 groups
    // 274 Mbit/s, 4 groups 270, 16 groups 272, 32 groups 268; fewer frames in
    // flight 212-248.
    int groups = o.groups > 0 ? o.groups : 2 * per_sm;
    int want_slots = o.max_active_frames;
    if (want_slots <= 0) {
        // frames in flight: about kStepBytes of algorithmic traffic (8E + 12n per
        // frame-iteration of the largest code, in FP32) per group step.  Measured at
        // n = 1e6 with 512 frames and 8 groups: 48 in flight 227.6 Mbit/s, 32: 225.8,
        // 64: 220.3, 96: 218.9, all 512: 200.4.  Small codes keep many more in flight.
        double bpf = 1.0;
        for (int c = 0; c < job.ngraphs; ++c)
            bpf = std::max(bpf, (8.0 * (double)job.graphs[c]->E + 12.0 * job.graphs[c]->n) * (sizeof(T) / 4.0));
        const long long per_group = std::max(1LL, (long long)std::ceil(kStepBytes / bpf));
        want_slots = (int)std::min<long long>(frames, per_group * std::max(1, std::min(groups, kMaxGroups)));
    }
    want_slots = std::min(std::min(want_slots, job.max_slot_frames), kMaxSlots);
    groups = std::max(1, std::min(std::min(groups, want_slots), std::min(grid, kMaxGroups)));
    const int slots_per_group = (want_slots + groups - 1) / groups;
    const int slots = groups * slots_per_group;
    grid = (grid / groups) * groups;
    const size_t smem = decode_smem_bytes(slots_per_group);

    // per-code sizes; slots are sized for the largest code
    CodeSet<Code> cs{};
    SlotSizes sz{};
    PackInfo pi{};
    code_set(job, grid / groups, slots_per_group, cs, sz, pi);
    const long long slot_E = sz.E;
    const int slot_n = sz.n, slot_nqb = sz.nqb, cn_max = sz.cn_max, vn_max = sz.vn_max;

    Layout L = make_layout(slots, sizeof(T), slot_E, slot_n, slot_nqb, job.sbits_words, o.debug_guards != 0);
    if (o.debug_guards) {
        L.guards.push_back(L.total);  // the guard after the last array
        L.total += kGuardBytes;
    }
    cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
    LDPC_TRY(cudaStreamIsCapturing(stream, &capturing));
    if (capturing != cudaStreamCaptureStatusNone && (ws.cap < L.total || !ws.ctrl))
        return LDPC_ERR_INVALID_ARG;  // run one decode of this size before capturing it
    ldpc_status st = ensure_workspace(ws, L.total);
    if (st != LDPC_OK) return st;
    char* base = (char*)ws.buf;
    ws.guard_off.clear();
    if (o.debug_guards) {
        st = fill_guards(ws, L.guards, stream);
        if (st != LDPC_OK) return st;
    }

    Params<T> p{};
    p.frames = frames;
    p.max_iter = job.max_iter;
    p.rule = job.rule;
    p.vnr_first_iter = o.vnr_first_iter;
    p.lmax = T(o.clamp);
    p.frame_code = job.frame_code;
    p.var_off = job.var_off;
    p.sb_off = job.sb_off;
    p.llr = job.llr;
    p.sbits = (const unsigned*)(base + L.sbits);
    p.bits_out = job.bits_out;
    p.flags_out = job.flags_out;
    p.iters_out = job.iters_out;
    p.slots = slots;
    p.slot_E = slot_E;
    p.slot_n = slot_n;
    p.slot_nqb = slot_nqb;
    p.cn_tiles_max = cn_max;
    p.vn_tiles_max = vn_max;
    p.c2v = (T*)(base + L.c2v);
    p.app = (T*)(base + L.app);
    p.qpart = (double*)(base + L.qpart);
    p.q0part = (double*)(base + L.q0part);
    p.qval = (double*)(base + L.qval);
    p.q0val = (double*)(base + L.q0val);
    p.unsat = (int*)(base + L.unsat);
    p.ctrl = ws.ctrl;
    p.trace_iters = o.trace_iters;
    p.trace_c2v = (T*)o.trace_c2v;
    p.trace_app = (T*)o.trace_app;
    p.trace_q = o.trace_q;
    p.timeout_ns = o.barrier_timeout_ms > 0 ? (unsigned long long)o.barrier_timeout_ms * 1000000ull
                                            : kBarrierTimeoutNs;
    p.bar_extra = o.test_unreachable_barrier ? 1u : 0u;
    p.groups = groups;
    p.slots_per_group = slots_per_group;
    p.new_frame = (int*)(base + L.new_frame);
    p.wts = job.wts;
    p.wcls = job.wcls;
    p.w_iters = job.w_iters;
    p.w_classes = job.w_classes;

    const bool timing = o.stats != nullptr && status_out == nullptr;
    if (timing) LDPC_TRY(cudaEventRecord(ws.ev[0], stream));
    // group barriers cleared; the queue of waiting frames starts after the first `slots`
    init_ctrl_kernel<<<1, 256, 0, stream>>>(ws.ctrl, groups, std::min(slots, frames), p.unsat, 2 * slots);
    LDPC_TRY(cudaGetLastError());
    {
        // about four words per warp; frames along y (grid-stride beyond 65535)
        int max_words = 1;
        for (int c = 0; c < job.ngraphs; ++c) max_words = std::max(max_words, pi.swords[c]);
        const dim3 pgrid((unsigned)std::min((max_words + 31) / 32, 4096), (unsigned)std::max(1, std::min(frames, 65535)));
        pack_syndrome_kernel<<<pgrid, 256, 0, stream>>>(job.syndrome, frames, pi, (unsigned*)(base + L.sbits),
                                                        ws.ctrl);
    }
    LDPC_TRY(cudaGetLastError());
    if (timing) LDPC_TRY(cudaEventRecord(ws.ev[1], stream));
    {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;  // all CTAs resident: the group barriers need it
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        LDPC_TRY(cudaLaunchKernelEx(&cfg, kernel, p, cs));
    }
    if (timing) LDPC_TRY(cudaEventRecord(ws.ev[2], stream));
    return finish_decode(ws, o, stream, status_out, grid, slots);
}

template <typename T, class Code>
ldpc_status launch_single(ldpc_graph* g, int frames, const float* llr, const uint8_t* syndrome, int max_iter,
                          int rule, uint8_t* bits_out, uint8_t* flags_out, int32_t* iters_out,
                          const ldpc_decode_opts& o, cudaStream_t stream, const float* wts = nullptr,
                          const int* wcls = nullptr, int w_iters = 0, int w_classes = 0) {
    const ldpc_graph* gs[1] = {g};
    Job job{};
    job.graphs = gs;
    job.ngraphs = 1;
    job.frames = frames;
    job.sbits_words = (long long)frames * ((g->m + 31) / 32);
    job.max_slot_frames = frames;
    job.llr = llr;
    job.syndrome = syndrome;
    job.bits_out = bits_out;
    job.flags_out = flags_out;
    job.iters_out = iters_out;
    job.max_iter = max_iter;
    job.rule = rule;
    job.wts = wts;
    job.wcls = wcls;
    job.w_iters = w_iters;
    job.w_classes = w_classes;
    return launch_decode<T, Code>(g->ws, job, o, stream);
}

ldpc_status check_decode_args(const ldpc_graph* graph, int32_t frames, const void* llr, const void* syndrome,
                              int32_t max_iter, int rule, const void* bits_out, const void* flags_out,
                              const void* iters_out, const ldpc_decode_opts& o) {
    if (!graph || frames < 0 || max_iter < 1 || rule < LDPC_TERM_NONE || rule > LDPC_TERM_PCE_VNR)
        return LDPC_ERR_INVALID_ARG;
    if (frames > 0 && (!llr || !syndrome || !bits_out || !flags_out || !iters_out)) return LDPC_ERR_INVALID_ARG;
    if (o.vnr_first_iter < 1 || !(o.clamp > 0.0f) || !std::isfinite(o.clamp)) return LDPC_ERR_INVALID_ARG;
    if (o.fp64 != 0 && o.fp64 != 1) return LDPC_ERR_INVALID_ARG;
    if (o.max_active_frames < 0 || o.max_active_frames > kMaxSlots || o.grid_ctas < 0 || o.trace_iters < 0 ||
        o.barrier_timeout_ms < 0 || o.groups < 0 || o.groups > kMaxGroups)
        return LDPC_ERR_INVALID_ARG;
    if (o.debug_guards != 0 && o.debug_guards != 1) return LDPC_ERR_INVALID_ARG;
    if (o.schedule < LDPC_SCHEDULE_AUTO || o.schedule > LDPC_SCHEDULE_FRAME_PAIR || o.flow_lag < 0 ||
        (o.schedule == LDPC_SCHEDULE_DATAFLOW && graph->kind != 1))
        return LDPC_ERR_INVALID_ARG;
    if ((long long)frames * graph->n > (1LL << 40)) return LDPC_ERR_INVALID_ARG;
    return LDPC_OK;
}

ldpc_status decode_weighted(const ldpc_graph* graph, int32_t frames, const float* llr, const uint8_t* syndrome,
                            int32_t max_iter, ldpc_term_rule rule, uint8_t* bits_out, uint8_t* flags_out,
                            int32_t* iters_out, const ldpc_decode_opts* opts, void* cuda_stream, const float* wts,
                            const int* wcls, int w_iters, int w_classes);

}  // namespace

extern "C" {

void ldpc_decode_opts_init(ldpc_decode_opts* opts) {
    if (!opts) return;
    std::memset(opts, 0, sizeof(*opts));
    opts->vnr_first_iter = 2;
    opts->clamp = 25.0f;
}

const char* ldpc_status_str(ldpc_status s) {
    switch (s) {
        case LDPC_OK: return "ok";
        case LDPC_ERR_INVALID_ARG: return "invalid argument";
        case LDPC_ERR_INVALID_GRAPH: return "invalid graph";
        case LDPC_ERR_OOM: return "out of memory";
        case LDPC_ERR_CUDA: return "CUDA error";
        case LDPC_ERR_TIMEOUT: return "grid synchronisation timed out";
        case LDPC_ERR_TOO_LARGE: return "problem too large for the fixed no-allocation scratch";
        case LDPC_ERR_BOUNDS: return "an index or guard check of the debug aids failed";
    }
    return "unknown status";
}

ldpc_status ldpc_graph_create_csr(int32_t m, int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                                  ldpc_graph** out) {
    if (!out) return LDPC_ERR_INVALID_ARG;
    *out = nullptr;
    if (m < 1 || n < 1 || !row_ptr) return LDPC_ERR_INVALID_ARG;
    if (row_ptr[0] != 0) return LDPC_ERR_INVALID_GRAPH;
    for (int32_t r = 0; r < m; ++r) {
        if (row_ptr[r + 1] < row_ptr[r]) return LDPC_ERR_INVALID_GRAPH;
        if (row_ptr[r + 1] - row_ptr[r] > kMaxDeg) return LDPC_ERR_INVALID_GRAPH;
    }
    const int64_t E = row_ptr[m];
    if (E > 0 && !col_idx) return LDPC_ERR_INVALID_ARG;
    std::vector<int> vdeg(n, 0);
    for (int32_t r = 0; r < m; ++r) {
        for (int32_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
            const int32_t v = col_idx[e];
            if (v < 0 || v >= n) return LDPC_ERR_INVALID_GRAPH;
            if (e > row_ptr[r] && col_idx[e - 1] >= v) return LDPC_ERR_INVALID_GRAPH;
            vdeg[v]++;
        }
    }
    std::vector<int> rp(row_ptr, row_ptr + m + 1), ci(col_idx, col_idx + E);
    std::vector<int> vp(n + 1, 0), ve(E);
    for (int v = 0; v < n; ++v) vp[v + 1] = vp[v] + vdeg[v];
    std::vector<int> fill(vp.begin(), vp.end() - 1);
    for (int64_t e = 0; e < E; ++e) ve[fill[ci[e]]++] = (int)e;  // ascending edge id per variable

    ldpc_graph* g = new (std::nothrow) ldpc_graph();
    if (!g) return LDPC_ERR_OOM;
    cudaError_t ce = cudaGetDevice(&g->device);
    if (ce != cudaSuccess) {
        delete g;
        return cuda_status(ce);
    }
    g->kind = 0;
    g->m = m;
    g->n = n;
    g->E = E;
    // checks ordered by degree (stable), so that the warps of a check pass that
    // walks this order meet one degree at a time
    std::vector<int> ro(m);
    for (int i = 0; i < m; ++i) ro[i] = i;
    std::stable_sort(ro.begin(), ro.end(), [&](int a, int b) { return rp[a + 1] - rp[a] < rp[b + 1] - rp[b]; });
    std::vector<const int*> d;
    ldpc_status st = upload_arrays({rp, ci, vp, ve, ro}, &g->dmem, d);
    if (st != LDPC_OK) {
        delete g;
        return st;
    }
    g->csr = CsrDev{m, n, d[0], d[1], d[2], d[3], d[4]};
    g->cn_tiles = (m + kCnTile - 1) / kCnTile;
    g->vn_tiles = (n + kVnTile - 1) / kVnTile;
    *out = g;
    return LDPC_OK;
}

ldpc_status ldpc_graph_create_qc(int32_t mb, int32_t nb, int32_t Z, const int32_t* shifts, ldpc_graph** out) {
    if (!out) return LDPC_ERR_INVALID_ARG;
    *out = nullptr;
    if (mb < 1 || nb < 1 || Z < 1 || !shifts) return LDPC_ERR_INVALID_ARG;
    if ((int64_t)mb * Z >= (1LL << 31) || (int64_t)nb * Z >= (1LL << 31)) return LDPC_ERR_INVALID_GRAPH;
    std::vector<int> row_ptr(mb + 1, 0), blk_col, blk_shift, col_cnt(nb, 0);
    for (int i = 0; i < mb; ++i) {
        for (int j = 0; j < nb; ++j) {
            const int32_t s = shifts[(int64_t)i * nb + j];
            if (s < -1 || s >= Z) return LDPC_ERR_INVALID_GRAPH;
            if (s >= 0) {
                blk_col.push_back(j);
                blk_shift.push_back(s);
                col_cnt[j]++;
            }
        }
        row_ptr[i + 1] = (int)blk_col.size();
        if (row_ptr[i + 1] - row_ptr[i] > kMaxDeg) return LDPC_ERR_INVALID_GRAPH;
    }
    const int nblk = (int)blk_col.size();
    if ((int64_t)nblk * Z >= (1LL << 31)) return LDPC_ERR_INVALID_GRAPH;
    std::vector<int> col_ptr(nb + 1, 0), col_blk(nblk), blk_row(nblk);
    for (int i = 0; i < mb; ++i)
        for (int b = row_ptr[i]; b < row_ptr[i + 1]; ++b) blk_row[b] = i;
    for (int j = 0; j < nb; ++j) col_ptr[j + 1] = col_ptr[j] + col_cnt[j];
    std::vector<int> fill(col_ptr.begin(), col_ptr.end() - 1);
    for (int b = 0; b < nblk; ++b) col_blk[fill[blk_col[b]]++] = b;  // row-major b => ascending row

    ldpc_graph* g = new (std::nothrow) ldpc_graph();
    if (!g) return LDPC_ERR_OOM;
    cudaError_t ce = cudaGetDevice(&g->device);
    if (ce != cudaSuccess) {
        delete g;
        return cuda_status(ce);
    }
    g->kind = 1;
    g->mb = mb;
    g->nb = nb;
    g->Z = Z;
    g->nblk = nblk;
    g->m = mb * Z;
    g->n = nb * Z;
    g->E = (int64_t)nblk * Z;
    std::vector<const int*> d;
    ldpc_status st = upload_arrays({row_ptr, blk_col, blk_shift, col_ptr, col_blk, blk_row}, &g->dmem, d);
    if (st != LDPC_OK) {
        delete g;
        return st;
    }
    g->qc = QcDev{mb, nb, Z, nblk, d[0], d[1], d[2], d[3], d[4], d[5]};
    g->h_row_ptr = row_ptr;
    g->h_blk_col = blk_col;
    g->h_blk_shift = blk_shift;
    g->h_col_ptr = col_ptr;
    g->h_col_blk = col_blk;
    g->h_blk_row = blk_row;
    g->row_deg.resize(mb);
    for (int i = 0; i < mb; ++i) g->row_deg[i] = row_ptr[i + 1] - row_ptr[i];
    g->col_deg.assign(col_cnt.begin(), col_cnt.end());
    g->cn_tiles = mb * ((Z + kQcCnChunk - 1) / kQcCnChunk);
    g->vn_tiles = nb * ((Z + kQcVnChunk - 1) / kQcVnChunk);
    *out = g;
    return LDPC_OK;
}

void ldpc_graph_destroy(ldpc_graph* g) {
    if (!g) return;
    DeviceGuard guard;
    guard.enter(g->device);
    free_workspace(g->ws);
    if (g->dmem) cudaFree(g->dmem);
    delete g;
}

ldpc_status ldpc_graph_info(const ldpc_graph* g, int32_t* m, int32_t* n, int64_t* edges) {
    if (!g) return LDPC_ERR_INVALID_ARG;
    if (m) *m = g->m;
    if (n) *n = g->n;
    if (edges) *edges = g->E;
    return LDPC_OK;
}

ldpc_status ldpc_decode(const ldpc_graph* graph, int32_t frames, const float* llr, const uint8_t* syndrome,
                        int32_t max_iter, ldpc_term_rule rule, uint8_t* bits_out, uint8_t* flags_out,
                        int32_t* iters_out, const ldpc_decode_opts* opts, void* cuda_stream) {
    NvtxRange nvtx("ldpc_decode");
    return decode_weighted(graph, frames, llr, syndrome, max_iter, rule, bits_out, flags_out, iters_out, opts,
                           cuda_stream, nullptr, nullptr, 0, 0);
}

ldpc_status ldpc_wbp_decode(const ldpc_wbp* plan, int32_t frames, const float* llr, const uint8_t* syndrome,
                            const float* weights, int32_t max_iter, ldpc_term_rule rule, uint8_t* bits_out,
                            uint8_t* flags_out, int32_t* iters_out, const ldpc_decode_opts* opts, void* cuda_stream) {
    NvtxRange nvtx("ldpc_wbp_decode");
    const ldpc_graph* graph = nullptr;
    const int* cls = nullptr;
    int iters = 0, classes = 0;
    if (!wbp_plan_classes(plan, &graph, &cls, &iters, &classes) || !weights) return LDPC_ERR_INVALID_ARG;
    return decode_weighted(graph, frames, llr, syndrome, max_iter, rule, bits_out, flags_out, iters_out, opts,
                           cuda_stream, weights, cls, iters, classes);
}

}  // extern "C"

namespace {

ldpc_status decode_weighted(const ldpc_graph* graph, int32_t frames, const float* llr, const uint8_t* syndrome,
                            int32_t max_iter, ldpc_term_rule rule, uint8_t* bits_out, uint8_t* flags_out,
                            int32_t* iters_out, const ldpc_decode_opts* opts, void* cuda_stream, const float* wts,
                            const int* wcls, int w_iters, int w_classes) {
    ldpc_decode_opts o;
    ldpc_decode_opts_init(&o);
    if (opts) o = *opts;
    ldpc_status st = check_decode_args(graph, frames, llr, syndrome, max_iter, (int)rule, bits_out, flags_out,
                                       iters_out, o);
    if (st != LDPC_OK) return st;
    if (o.trace_iters > 0 && !o.trace_c2v && !o.trace_app && !o.trace_q) o.trace_iters = 0;
    if (frames == 0) {
        if (o.stats) std::memset(o.stats, 0, sizeof(*o.stats));
        return LDPC_OK;
    }
    ldpc_graph* g = const_cast<ldpc_graph*>(graph);
    DeviceGuard guard;
    LDPC_TRY(guard.enter(g->device));
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    if (g->kind == 1) {
        if (o.fp64)
            return launch_single<double, QcDev>(g, frames, llr, syndrome, max_iter, (int)rule, bits_out, flags_out,
                                                iters_out, o, stream, wts, wcls, w_iters, w_classes);
        return launch_single<float, QcDev>(g, frames, llr, syndrome, max_iter, (int)rule, bits_out, flags_out,
                                           iters_out, o, stream, wts, wcls, w_iters, w_classes);
    }
    if (o.fp64)
        return launch_single<double, CsrDev>(g, frames, llr, syndrome, max_iter, (int)rule, bits_out, flags_out,
                                             iters_out, o, stream, wts, wcls, w_iters, w_classes);
    return launch_single<float, CsrDev>(g, frames, llr, syndrome, max_iter, (int)rule, bits_out, flags_out,
                                        iters_out, o, stream, wts, wcls, w_iters, w_classes);
}

}  // namespace

extern "C" {

ldpc_status ldpc_decode_host(const ldpc_graph* graph, int32_t frames, const float* llr, const uint8_t* syndrome,
                             int32_t max_iter, ldpc_term_rule rule, uint8_t* bits_out, uint8_t* flags_out,
                             int32_t* iters_out, const ldpc_decode_opts* opts, void* cuda_stream) {
    NvtxRange nvtx("ldpc_decode_host");
    ldpc_decode_opts o;
    ldpc_decode_opts_init(&o);
    if (opts) o = *opts;
    ldpc_status st = check_decode_args(graph, frames, llr, syndrome, max_iter, (int)rule, bits_out, flags_out,
                                       iters_out, o);
    if (st != LDPC_OK) return st;
    if (o.trace_c2v || o.trace_app || o.trace_q) return LDPC_ERR_INVALID_ARG;
    if (frames == 0) return LDPC_OK;
    ldpc_graph* g = const_cast<ldpc_graph*>(graph);
    DeviceGuard guard;
    LDPC_TRY(guard.enter(g->device));
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    const size_t n_llr = (size_t)frames * g->n * sizeof(float);
    const size_t n_syn = (size_t)frames * g->m;
    const size_t n_bits = (size_t)frames * g->n;
    const size_t o_syn = align_up(n_llr, 256), o_bits = o_syn + align_up(n_syn, 256);
    const size_t o_flags = o_bits + align_up(n_bits, 256), o_iters = o_flags + align_up((size_t)frames, 256);
    const size_t total = o_iters + align_up((size_t)frames * sizeof(int32_t), 256);
    Workspace& ws = g->ws;
    if (ws.stage_cap < total) {
        if (ws.stage) cudaFree(ws.stage);
        ws.stage = nullptr;
        ws.stage_cap = 0;
        LDPC_TRY(cudaMalloc(&ws.stage, total));
        ws.stage_cap = total;
    }
    char* d = (char*)ws.stage;
    LDPC_TRY(cudaMemcpyAsync(d, llr, n_llr, cudaMemcpyHostToDevice, stream));
    LDPC_TRY(cudaMemcpyAsync(d + o_syn, syndrome, n_syn, cudaMemcpyHostToDevice, stream));
    st = ldpc_decode(graph, frames, (const float*)d, (const uint8_t*)(d + o_syn), max_iter, rule,
                     (uint8_t*)(d + o_bits), (uint8_t*)(d + o_flags), (int32_t*)(d + o_iters), &o, cuda_stream);
    if (st != LDPC_OK) return st;
    LDPC_TRY(cudaMemcpyAsync(bits_out, d + o_bits, n_bits, cudaMemcpyDeviceToHost, stream));
    LDPC_TRY(cudaMemcpyAsync(flags_out, d + o_flags, (size_t)frames, cudaMemcpyDeviceToHost, stream));
    LDPC_TRY(cudaMemcpyAsync(iters_out, d + o_iters, (size_t)frames * sizeof(int32_t), cudaMemcpyDeviceToHost,
                             stream));
    LDPC_TRY(cudaStreamSynchronize(stream));
    return LDPC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches of frames of several codes (ldpc_batch_*).
// ---------------------------------------------------------------------------
struct ldpc_batch {
    std::vector<const ldpc_graph*> graphs;
    int kind = 0, device = 0, frames = 0, max_slot_frames = 0;
    void* dmem = nullptr;            // frame_code | var_off | syn_off | sb_off
    const int* frame_code = nullptr;
    const long long* var_off = nullptr;
    const long long* syn_off = nullptr;
    const long long* sb_off = nullptr;
    long long llr_len = 0, syn_len = 0, sb_words = 0;
    bool var_unaligned[kMaxCodes] = {};     // a frame of code c starts at an offset not a multiple of 4
    int tuned_groups = 0, tuned_slots = 0;  // from ldpc_batch_autotune (0 = none)
    int tuned_cn[kMaxCodes] = {}, tuned_vn[kMaxCodes] = {};  // QC item sizes per code (0 = model's pick)
    Workspace ws;
};

namespace {

ldpc_decode_opts batch_opts(const ldpc_batch* b, const ldpc_decode_opts* opts) {
    ldpc_decode_opts o;
    ldpc_decode_opts_init(&o);
    if (opts) o = *opts;
    if (o.groups == 0) o.groups = b->tuned_groups;
    if (o.max_active_frames == 0) o.max_active_frames = b->tuned_slots;
    return o;
}

ldpc_status batch_launch(ldpc_batch* b, const float* llr, const uint8_t* syndrome, int32_t max_iter,
                         ldpc_term_rule rule, uint8_t* bits_out, uint8_t* flags_out, int32_t* iters_out,
                         const ldpc_decode_opts& o, cudaStream_t stream, int32_t* status_out) {
    Job job{};
    job.graphs = b->graphs.data();
    job.ngraphs = (int)b->graphs.size();
    job.frames = b->frames;
    job.frame_code = b->frame_code;
    job.var_off = b->var_off;
    job.syn_off = b->syn_off;
    job.sb_off = b->sb_off;
    job.sbits_words = b->sb_words;
    job.max_slot_frames = b->max_slot_frames;
    job.llr = llr;
    job.syndrome = syndrome;
    job.bits_out = bits_out;
    job.flags_out = flags_out;
    job.iters_out = iters_out;
    job.max_iter = max_iter;
    job.rule = (int)rule;
    for (int c = 0; c < kMaxCodes; ++c) {
        job.var_unaligned[c] = b->var_unaligned[c];
        job.cn_chunk[c] = b->tuned_cn[c];
        job.vn_chunk[c] = b->tuned_vn[c];
    }
    if (b->kind == 1) {
        if (o.fp64) return launch_decode<double, QcDev>(b->ws, job, o, stream, status_out);
        return launch_decode<float, QcDev>(b->ws, job, o, stream, status_out);
    }
    if (o.fp64) return launch_decode<double, CsrDev>(b->ws, job, o, stream, status_out);
    return launch_decode<float, CsrDev>(b->ws, job, o, stream, status_out);
}

ldpc_status check_batch_args(const ldpc_batch* b, const void* llr, const void* syndrome, int32_t max_iter,
                             int rule, const void* bits, const void* flags, const void* iters,
                             const ldpc_decode_opts& o) {
    if (!b) return LDPC_ERR_INVALID_ARG;
    if (o.trace_iters > 0 || o.trace_c2v || o.trace_app || o.trace_q) return LDPC_ERR_INVALID_ARG;
    return check_decode_args(b->graphs[0], b->frames, llr, syndrome, max_iter, rule, bits, flags, iters, o);
}

}  // namespace

extern "C" {

ldpc_status ldpc_batch_create(const ldpc_graph* const* graphs, int32_t n_graphs, int32_t frames,
                              const int32_t* frame_graph, ldpc_batch** out) {
    if (!out) return LDPC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!graphs || n_graphs < 1 || n_graphs > kMaxCodes || frames < 1 || !frame_graph) return LDPC_ERR_INVALID_ARG;
    for (int c = 0; c < n_graphs; ++c) {
        if (!graphs[c] || graphs[c]->kind != graphs[0]->kind || graphs[c]->device != graphs[0]->device)
            return LDPC_ERR_INVALID_ARG;
    }
    std::vector<int> code(frames);
    std::vector<long long> var_off(frames), syn_off(frames), sb_off(frames);
    long long vo = 0, so = 0, wo = 0;
    for (int f = 0; f < frames; ++f) {
        const int c = frame_graph[f];
        if (c < 0 || c >= n_graphs) return LDPC_ERR_INVALID_ARG;
        code[f] = c;
        var_off[f] = vo;
        syn_off[f] = so;
        sb_off[f] = wo;
        vo += graphs[c]->n;
        so += graphs[c]->m;
        wo += (graphs[c]->m + 31) / 32;
    }
    ldpc_batch* b = new (std::nothrow) ldpc_batch();
    if (!b) return LDPC_ERR_OOM;
    b->graphs.assign(graphs, graphs + n_graphs);
    b->kind = graphs[0]->kind;
    b->device = graphs[0]->device;
    b->frames = frames;
    b->max_slot_frames = frames;
    b->llr_len = vo;
    b->syn_len = so;
    b->sb_words = wo;
    for (int f = 0; f < frames; ++f)
        if (var_off[f] % 4 != 0) b->var_unaligned[code[f]] = true;
    DeviceGuard guard;
    cudaError_t ce = guard.enter(b->device);
    const size_t bytes = align_up((size_t)frames * sizeof(int), 256) + 3 * align_up((size_t)frames * 8, 256);
    if (ce == cudaSuccess) ce = cudaMalloc(&b->dmem, bytes);
    if (ce != cudaSuccess) {
        delete b;
        return cuda_status(ce);
    }
    char* d = (char*)b->dmem;
    const size_t o1 = align_up((size_t)frames * sizeof(int), 256), ob = align_up((size_t)frames * 8, 256);
    b->frame_code = (const int*)d;
    b->var_off = (const long long*)(d + o1);
    b->syn_off = (const long long*)(d + o1 + ob);
    b->sb_off = (const long long*)(d + o1 + 2 * ob);
    ce = cudaMemcpy(d, code.data(), (size_t)frames * sizeof(int), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(d + o1, var_off.data(), (size_t)frames * 8, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(d + o1 + ob, syn_off.data(), (size_t)frames * 8, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess)
        ce = cudaMemcpy(d + o1 + 2 * ob, sb_off.data(), (size_t)frames * 8, cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) {
        cudaFree(b->dmem);
        delete b;
        return cuda_status(ce);
    }
    *out = b;
    return LDPC_OK;
}

void ldpc_batch_destroy(ldpc_batch* b) {
    if (!b) return;
    DeviceGuard guard;
    guard.enter(b->device);
    free_workspace(b->ws);
    if (b->dmem) cudaFree(b->dmem);
    delete b;
}

ldpc_status ldpc_batch_info(const ldpc_batch* b, int32_t* frames, int64_t* llr_len, int64_t* syndrome_len) {
    if (!b) return LDPC_ERR_INVALID_ARG;
    if (frames) *frames = b->frames;
    if (llr_len) *llr_len = b->llr_len;
    if (syndrome_len) *syndrome_len = b->syn_len;
    return LDPC_OK;
}

ldpc_status ldpc_batch_decode(ldpc_batch* b, const float* llr, const uint8_t* syndrome, int32_t max_iter,
                              ldpc_term_rule rule, uint8_t* bits_out, uint8_t* flags_out, int32_t* iters_out,
                              const ldpc_decode_opts* opts, void* cuda_stream) {
    NvtxRange nvtx("ldpc_batch_decode");
    if (!b) return LDPC_ERR_INVALID_ARG;
    const ldpc_decode_opts o = batch_opts(b, opts);
    ldpc_status st = check_batch_args(b, llr, syndrome, max_iter, (int)rule, bits_out, flags_out, iters_out, o);
    if (st != LDPC_OK) return st;
    DeviceGuard guard;
    LDPC_TRY(guard.enter(b->device));
    return batch_launch(b, llr, syndrome, max_iter, rule, bits_out, flags_out, iters_out, o,
                        (cudaStream_t)cuda_stream, nullptr);
}

ldpc_status ldpc_batch_decode_async(ldpc_batch* b, const float* llr, const uint8_t* syndrome, int32_t max_iter,
                                    ldpc_term_rule rule, uint8_t* bits_out, uint8_t* flags_out, int32_t* iters_out,
                                    int32_t* status_out, const ldpc_decode_opts* opts, void* cuda_stream) {
    NvtxRange nvtx("ldpc_batch_decode_async");
    if (!b || !status_out) return LDPC_ERR_INVALID_ARG;
    ldpc_decode_opts o = batch_opts(b, opts);
    o.stats = nullptr;
    ldpc_status st = check_batch_args(b, llr, syndrome, max_iter, (int)rule, bits_out, flags_out, iters_out, o);
    if (st != LDPC_OK) return st;
    DeviceGuard guard;
    LDPC_TRY(guard.enter(b->device));
    return batch_launch(b, llr, syndrome, max_iter, rule, bits_out, flags_out, iters_out, o,
                        (cudaStream_t)cuda_stream, status_out);
}

ldpc_status ldpc_batch_autotune(ldpc_batch* b, const float* llr, const uint8_t* syndrome, int32_t max_iter,
                                ldpc_term_rule rule, uint8_t* bits_out, uint8_t* flags_out, int32_t* iters_out,
                                void* cuda_stream, int32_t* best_groups, int32_t* best_slots) {
    NvtxRange nvtx("ldpc_batch_autotune");
    if (!b) return LDPC_ERR_INVALID_ARG;
    ldpc_decode_opts o;
    ldpc_decode_opts_init(&o);
    ldpc_status st = check_batch_args(b, llr, syndrome, max_iter, (int)rule, bits_out, flags_out, iters_out, o);
    if (st != LDPC_OK) return st;
    DeviceGuard guard;
    LDPC_TRY(guard.enter(b->device));
    int dev = 0, per_sm = 0;
    LDPC_TRY(cudaGetDevice(&dev));
    LDPC_TRY(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMultiProcessorCount, dev));
    // candidates: groups in {1, 2, 4, 8}; slots in {all frames, 8 per group, 2 per group}
    const int F = std::min(b->frames, kMaxSlots);
    float best_ms = -1.0f;
    int bg = 0, bs = 0;
    for (int c = 0; c < kMaxCodes; ++c) b->tuned_cn[c] = b->tuned_vn[c] = 0;  // start from the model
    // one untimed decode at the largest slot count first: sizes the workspace
    // and warms caches and clocks, so the first candidate is not timed cold
    o.groups = 1;
    o.max_active_frames = F;
    st = batch_launch(b, llr, syndrome, max_iter, rule, bits_out, flags_out, iters_out, o, (cudaStream_t)cuda_stream,
                      nullptr);
    if (st != LDPC_OK) return st;
    const int gcand[] = {1, 2, 4, 8};
    for (int gi = 0; gi < 4; ++gi) {
        const int gcount = gcand[gi];
        const int scand[] = {F, std::min(F, 8 * gcount), std::min(F, 2 * gcount)};
        for (int si = 0; si < 3; ++si) {
            if (si > 0 && scand[si] == scand[si - 1]) continue;
            ldpc_decode_stats stats{};
            o.groups = gcount;
            o.max_active_frames = scand[si];
            o.stats = &stats;
            st = batch_launch(b, llr, syndrome, max_iter, rule, bits_out, flags_out, iters_out, o,
                              (cudaStream_t)cuda_stream, nullptr);
            if (st != LDPC_OK) return st;
            if (best_ms < 0.0f || stats.kernel_ms < best_ms) {
                best_ms = stats.kernel_ms;
                bg = gcount;
                bs = scand[si];
            }
        }
    }
    b->tuned_groups = bg;
    b->tuned_slots = bs;
    // then, per QC code, its item sizes (check side, then variable side) by
    // coordinate descent from the model's pick, with the block schedule fixed
    if (b->kind == 1) {
        static const int cn_cand[] = {512, 1024, 2048, 4096};
        static const int vn_cand[] = {1024, 2048, 4096, 8192};
        o.groups = bg;
        o.max_active_frames = bs;
        for (int c = 0; c < (int)b->graphs.size(); ++c) {
            for (int side = 0; side < 2; ++side) {
                int* slot = side == 0 ? &b->tuned_cn[c] : &b->tuned_vn[c];
                const int* cand = side == 0 ? cn_cand : vn_cand;
                int keep = 0;  // 0: the model's pick, timed first
                for (int ci = -1; ci < 4; ++ci) {
                    *slot = ci < 0 ? 0 : cand[ci];
                    ldpc_decode_stats stats{};
                    o.stats = &stats;
                    st = batch_launch(b, llr, syndrome, max_iter, rule, bits_out, flags_out, iters_out, o,
                                      (cudaStream_t)cuda_stream, nullptr);
                    if (st != LDPC_OK) return st;
                    if (stats.kernel_ms < best_ms) {
                        best_ms = stats.kernel_ms;
                        keep = *slot;
                    }
                }
                *slot = keep;
            }
        }
    }
    if (best_groups) *best_groups = bg;
    if (best_slots) *best_slots = bs;
    return LDPC_OK;
}

ldpc_status ldpc_graph_check_guards(const ldpc_graph* graph) {
    if (!graph) return LDPC_ERR_INVALID_ARG;
    return check_guards(const_cast<ldpc_graph*>(graph)->ws, graph->device);
}

ldpc_status ldpc_batch_check_guards(const ldpc_batch* batch) {
    if (!batch) return LDPC_ERR_INVALID_ARG;
    return check_guards(const_cast<ldpc_batch*>(batch)->ws, batch->device);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Entry point that allocates nothing: ldpc_decode_qc_noalloc.
//
// For callers that must not allocate device memory (real-time loops that
// cannot pay for cudaMalloc/cudaFree, hosts whose memory manager owns the
// GPU's memory).  All device state lives in one file-scope array; the host
// side only copies the QC tables in, clears the control words and launches
// the same two kernels ldpc_decode uses.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoallocBytes = LDPC_NOALLOC_SCRATCH_BYTES;
constexpr int kNoallocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kNoallocMaxDevices] = {};

// Device address of the scratch on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device with that device current.
ldpc_status noalloc_scratch(int dev, char** out) {
    if (dev < 0 || dev >= kNoallocMaxDevices) return LDPC_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || ptr == nullptr) return cuda_status(e == cudaSuccess ? cudaErrorUnknown : e);
        g_noalloc_addr[dev] = ptr;
    }
    *out = (char*)g_noalloc_addr[dev];
    return LDPC_OK;
}

struct NoallocLayout {
    size_t ctrl, tables, sbits, unsat, qval, q0val, qpart, q0part, new_frame, c2v, app, total;
    int slots;
};

// Carve the scratch for `slots` concurrent frames; total > kNoallocBytes means it does not fit.
NoallocLayout noalloc_layout(size_t table_ints, int64_t n, int64_t E, int nqb, int frames, int swords,
                             int slots) {
    NoallocLayout L{};
    size_t o = 0;
    L.ctrl = o;   o = align_up(o + sizeof(Ctrl), 256);
    L.tables = o; o = align_up(o + table_ints * sizeof(int), 256);
    L.sbits = o;  o = align_up(o + (size_t)frames * swords * sizeof(unsigned), 256);
    L.unsat = o;  o = align_up(o + 2 * (size_t)slots * sizeof(int), 256);
    L.qval = o;   o = align_up(o + (size_t)slots * kQParts * sizeof(double), 256);
    L.q0val = o;  o = align_up(o + (size_t)slots * kQParts * sizeof(double), 256);
    L.qpart = o;  o = align_up(o + (size_t)slots * nqb * kWarps * sizeof(double), 256);
    L.q0part = o; o = align_up(o + (size_t)slots * nqb * kWarps * sizeof(double), 256);
    L.new_frame = o; o = align_up(o + (size_t)slots * sizeof(int), 256);
    L.c2v = o;    o = align_up(o + (size_t)slots * (size_t)E * sizeof(float), 256);
    L.app = o;    o = align_up(o + (size_t)slots * (size_t)n * sizeof(float), 256);
    L.total = o;
    L.slots = slots;
    return L;
}

}  // namespace

extern "C" ldpc_status ldpc_decode_qc_noalloc(int32_t mb, int32_t nb, int32_t Z, const int32_t* shifts,
                                              int32_t frames, const float* llr, const uint8_t* syndrome,
                                              int32_t max_iter, ldpc_term_rule rule, uint8_t* bits_out,
                                              uint8_t* flags_out, int32_t* iters_out, void* cuda_stream) {
    // ---- host-side checks (nothing queued yet) ----
    if (mb < 1 || nb < 1 || Z < 1 || !shifts) return LDPC_ERR_INVALID_ARG;
    if (frames < 0 || max_iter < 1 || (int)rule < LDPC_TERM_NONE || (int)rule > LDPC_TERM_PCE_VNR)
        return LDPC_ERR_INVALID_ARG;
    if (frames > 0 && (!llr || !syndrome || !bits_out || !flags_out || !iters_out)) return LDPC_ERR_INVALID_ARG;
    if ((int64_t)mb * Z >= (1LL << 31) || (int64_t)nb * Z >= (1LL << 31)) return LDPC_ERR_INVALID_GRAPH;
    std::vector<int> row_ptr(mb + 1, 0), blk_col, blk_shift, col_cnt(nb, 0);
    for (int i = 0; i < mb; ++i) {
        for (int j = 0; j < nb; ++j) {
            const int32_t sv = shifts[(int64_t)i * nb + j];
            if (sv < -1 || sv >= Z) return LDPC_ERR_INVALID_GRAPH;
            if (sv >= 0) {
                blk_col.push_back(j);
                blk_shift.push_back(sv);
                col_cnt[j]++;
            }
        }
        row_ptr[i + 1] = (int)blk_col.size();
        if (row_ptr[i + 1] - row_ptr[i] > kMaxDeg) return LDPC_ERR_INVALID_GRAPH;
    }
    const int nblk = (int)blk_col.size();
    if ((int64_t)nblk * Z >= (1LL << 31)) return LDPC_ERR_INVALID_GRAPH;
    std::vector<int> col_ptr(nb + 1, 0), col_blk(nblk), blk_row(nblk);
    for (int i = 0; i < mb; ++i)
        for (int b = row_ptr[i]; b < row_ptr[i + 1]; ++b) blk_row[b] = i;
    for (int j = 0; j < nb; ++j) col_ptr[j + 1] = col_ptr[j] + col_cnt[j];
    {
        std::vector<int> fill(col_ptr.begin(), col_ptr.end() - 1);
        for (int b = 0; b < nblk; ++b) col_blk[fill[blk_col[b]]++] = b;
    }
    // one host table, uploaded in one copy: row_ptr | blk_col | blk_shift | col_ptr | col_blk | blk_row
    std::vector<int> table;
    table.reserve((size_t)(mb + 1) + 4 * (size_t)nblk + (size_t)(nb + 1));
    size_t off[6];
    const std::vector<int>* parts[6] = {&row_ptr, &blk_col, &blk_shift, &col_ptr, &col_blk, &blk_row};
    for (int k = 0; k < 6; ++k) {
        off[k] = table.size();
        table.insert(table.end(), parts[k]->begin(), parts[k]->end());
    }
    const int32_t m = mb * Z, n = nb * Z;
    const int64_t E = (int64_t)nblk * Z;
    const int swords = (m + 31) / 32;
    const int vn_tiles = nb * ((Z + kQcVnChunk - 1) / kQcVnChunk);
    const int cn_tiles = mb * ((Z + kQcCnChunk - 1) / kQcCnChunk);
    const int nqb = nb * ((Z + kQBlock - 1) / kQBlock);
    if (frames == 0) return LDPC_OK;
    int slots = std::min(frames, kMaxSlots);
    while (slots > 0 && noalloc_layout(table.size(), n, E, nqb, frames, swords, slots).total > kNoallocBytes)
        --slots;
    if (slots < 1) return LDPC_ERR_TOO_LARGE;
    const NoallocLayout L = noalloc_layout(table.size(), n, E, nqb, frames, swords, slots);

    // ---- device work, all inside the fixed scratch ----
    int dev = 0, sms = 0, per_sm = 0, coop = 0;
    LDPC_TRY(cudaGetDevice(&dev));
    char* base = nullptr;
    ldpc_status st = noalloc_scratch(dev, &base);
    if (st != LDPC_OK) return st;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    LDPC_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    LDPC_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (!coop) return LDPC_ERR_CUDA;
    auto kernel = bp_decode_kernel<float, QcDev, false>;
    // one group holds every slot: the same per-slot table as ldpc_decode's launches
    const size_t smem = decode_smem_bytes(slots);
    LDPC_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)decode_smem_bytes(kMaxSlots)));
    LDPC_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, smem));
    if (per_sm < 1) return LDPC_ERR_CUDA;
    const int grid = std::min(per_sm * sms, kMaxGrid);

    int* dtab = (int*)(base + L.tables);
    LDPC_TRY(cudaMemcpyAsync(dtab, table.data(), table.size() * sizeof(int), cudaMemcpyHostToDevice, stream));
    const QcDev code{mb, nb, Z, nblk, dtab + off[0], dtab + off[1], dtab + off[2], dtab + off[3], dtab + off[4],
                     dtab + off[5]};
    Ctrl* ctrl = (Ctrl*)(base + L.ctrl);
    Ctrl c0{};
    c0.next_frame = std::min(slots, frames);  // the queue of waiting frames starts after the slots
    LDPC_TRY(cudaMemcpyAsync(ctrl, &c0, sizeof(Ctrl), cudaMemcpyHostToDevice, stream));
    LDPC_TRY(cudaMemsetAsync(base + L.unsat, 0, 2 * (size_t)slots * sizeof(int), stream));

    CodeSet<QcDev> cs{};
    cs.count = 1;
    CodeInfo<QcDev>& ci = cs.c[0];
    ci.code = code;
    ci.n = n;
    ci.m = m;
    ci.E = E;
    ci.swords = swords;
    ci.cn_tiles = cn_tiles;
    ci.vn_tiles = vn_tiles;
    ci.cn_chunk = kQcCnChunk;
    ci.vn_chunk = kQcVnChunk;
    ci.nqb = nqb;
    ci.vec4 = ((Z % 4) == 0 && ((uintptr_t)llr % 16) == 0) ? 1 : 0;

    Params<float> p{};
    p.frames = frames;
    p.max_iter = max_iter;
    p.rule = (int)rule;
    p.vnr_first_iter = 2;
    p.lmax = 25.0f;
    p.llr = llr;
    p.sbits = (const unsigned*)(base + L.sbits);
    p.bits_out = bits_out;
    p.flags_out = flags_out;
    p.iters_out = iters_out;
    p.slots = slots;
    p.slot_E = E;
    p.slot_n = n;
    p.slot_nqb = nqb;
    p.cn_tiles_max = cn_tiles;
    p.vn_tiles_max = vn_tiles;
    p.c2v = (float*)(base + L.c2v);
    p.app = (float*)(base + L.app);
    p.qpart = (double*)(base + L.qpart);
    p.q0part = (double*)(base + L.q0part);
    p.qval = (double*)(base + L.qval);
    p.q0val = (double*)(base + L.q0val);
    p.unsat = (int*)(base + L.unsat);
    p.ctrl = ctrl;
    p.trace_iters = 0;
    p.timeout_ns = kBarrierTimeoutNs;
    p.groups = 1;
    p.slots_per_group = slots;
    p.new_frame = (int*)(base + L.new_frame);
    {
        PackInfo pi{};
        pi.m[0] = m;
        pi.swords[0] = swords;
        const dim3 pgrid((unsigned)std::max(1, std::min((swords + 31) / 32, 4096)), (unsigned)std::max(1, std::min(frames, 65535)));
        pack_syndrome_kernel<<<pgrid, 256, 0, stream>>>(syndrome, frames, pi, (unsigned*)(base + L.sbits), ctrl);
        LDPC_TRY(cudaGetLastError());
    }
    void* args[] = {(void*)&p, (void*)&cs};
    LDPC_TRY(cudaLaunchCooperativeKernel((const void*)kernel, dim3(grid), dim3(kThreads), args, smem, stream));
    int err = 0;
    LDPC_TRY(cudaMemcpyAsync(&err, &ctrl->err, sizeof(int), cudaMemcpyDeviceToHost, stream));
    LDPC_TRY(cudaStreamSynchronize(stream));
    if (err == kErrSyndrome) return LDPC_ERR_INVALID_ARG;
    if (err == kErrTimeout) return LDPC_ERR_TIMEOUT;
    if (err == kErrBounds) return LDPC_ERR_BOUNDS;
    if (err != kErrNone) return LDPC_ERR_CUDA;
    return LDPC_OK;
}

