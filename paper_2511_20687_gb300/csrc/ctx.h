// Host runtime of libosam, shared by its translation units: the context of a problem or a batch of
// instances (groups of FOM / ROM subdomains across instances, couplings, controller state, graphs,
// streams, profiling), the checked-call macros and the functions one unit calls in another.
// Internal: only setup.cu, controller.cu and osam_api.cu include it.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "osam.h"
#include "osam_internal.h"

namespace osam {
namespace host {

struct FomGroupH {
    std::vector<Grid> grid;
    std::vector<std::vector<uint8_t>> clamp;
    std::vector<std::vector<int>> srow;
    std::vector<int> ns;
    std::vector<InstFom> inst;
    std::vector<int> nblk_off;
    std::vector<int2> nblk;
    FomB d{};
    InstFom* inst_d = nullptr;
};

struct RomGroupH {
    std::vector<Grid> grid;
    std::vector<std::vector<uint8_t>> clamp;
    std::vector<std::vector<int>> srow;
    std::vector<int> ns, nfree;
    std::vector<InstRom> inst;
    // per-instance device pointers into flat arrays (set-up / I/O)
    std::vector<double*> Phi;
    std::vector<int*> free_dof, dof_free, srow_d;
    std::vector<uint8_t*> clamp_d;
    RomB d{};
    InstRom* inst_d = nullptr;
};

struct Slot {
    int kind = OSAM_FOM;
    int nsub = 0;        // substeps per controller interval (Sec. 4.1: n_i)
    double dt = 0.0;     // Delta t_i = interval length / n_i
    FomGroupH fom;
    RomGroupH rom;
};

struct CplH {
    int dst = 0, src = 0;
    std::vector<int> nrow, row_first;
    CplB d{};
};

}  // namespace host
}  // namespace osam

// the runtime's units are written against the library's own namespaces
using namespace osam;
using namespace osam::host;

struct osam_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int n_inst = 1;
    double dt = 0.0;
    int nsub = 0;
    double tol_abs = 0.0, tol_rel = 0.0;
    int max_it = 1;
    int precision = OSAM_FP64;
    int scatter = kGather;
    std::vector<Slot> slots;
    std::vector<CplH> cpls;
    std::vector<void*> allocs;
    std::vector<long long> fom_elements;  // per instance
    CtlB ctl{};
    int* sel = nullptr;                   // one-hot instance mask for per-instance I/O
    int* iters_h = nullptr;               // pinned mirrors
    int* status_h = nullptr;
    double* cnum_h = nullptr;
    double* cden_h = nullptr;
    int* any_h = nullptr;
    int* imp_h = nullptr;                 // pinned mirror of a per-instance Newton / CG activity mask
    bool any_implicit = false;            // some FOM group integrates implicitly
    // implicit intervals as CUDA graphs with device-side Newton / CG loops: two streams on which the
    // bodies of the nested conditional nodes are captured, and one instantiated interval per
    // (subdomain, activity mask) for launches outside a controller-step capture
    cudaStream_t cap[2] = {nullptr, nullptr};
    struct ImpExec {
        int slot;
        const int* active;
        cudaGraph_t graph;
        cudaGraphExec_t exec;
        long long kernels;
    };
    std::vector<ImpExec> imp_exec;
    double* scratch = nullptr;            // device [3 * max nodes of any instance]
    int* err_d = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // side stream that advances a ROM subdomain one substep behind the FOM that feeds it, joined back
    // with events (also inside the graph capture).  It has the lowest priority, so its small kernels
    // take the SM slots the internal-force kernel leaves free in its last wave instead of delaying it.
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // additive Schwarz: every subdomain but the first advances on a stream of its own, forked from and
    // joined back to the context stream in every iteration (also inside the graph capture)
    bool additive = false;
    std::vector<cudaStream_t> lanes;
    std::vector<cudaEvent_t> lane_join;
    std::string err;
    // CUDA graph of one controller step: begin nodes, then a while node over Schwarz iterations
    bool use_graph = true;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle cond{};
    long long graph_begin_launches = 0, graph_body_launches = 0;  // kernels per graph part (counted at capture)
    // kernel-level timing of the internal-force launches (host-driven path) and a launch count
    bool prof = false;
    std::vector<cudaEvent_t> pev;
    std::vector<int> pkind;               // per event pair: 0 internal force, 1 implicit tangent action
    int pnext = 0;
    double prof_ms = 0.0, tprof_ms = 0.0;
    long long prof_launches = 0, prof_elements = 0, launches = 0;
    long long tprof_launches = 0;

    ~osam_ctx() {
        if (stream) cudaStreamSynchronize(stream);
        if (side) cudaStreamSynchronize(side);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (void* p : allocs) cudaFree(p);
        if (iters_h) cudaFreeHost(iters_h);
        if (status_h) cudaFreeHost(status_h);
        if (cnum_h) cudaFreeHost(cnum_h);
        if (cden_h) cudaFreeHost(cden_h);
        if (any_h) cudaFreeHost(any_h);
        if (imp_h) cudaFreeHost(imp_h);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        for (cudaEvent_t e : pev) cudaEventDestroy(e);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        for (ImpExec& x : imp_exec) {
            cudaGraphExecDestroy(x.exec);
            cudaGraphDestroy(x.graph);
        }
        for (cudaStream_t c : cap)
            if (c) cudaStreamDestroy(c);
        for (cudaEvent_t e : lane_join) cudaEventDestroy(e);
        for (cudaStream_t l : lanes) {
            cudaStreamSynchronize(l);
            cudaStreamDestroy(l);
        }
        if (side) cudaStreamDestroy(side);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }

    template <typename T>
    T* alloc(size_t n) {
        if (n == 0) n = 1;
        void* p = nullptr;
        if (cudaMalloc(&p, n * sizeof(T)) != cudaSuccess) return nullptr;
        allocs.push_back(p);
        cudaMemsetAsync(p, 0, n * sizeof(T), stream);
        return static_cast<T*>(p);
    }

    int fail(int code, const char* fmt, ...) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        err = buf;
        return code;
    }

    int prof_begin(int kind = 0) {
        if (!prof) return -1;
        while (pnext + 2 > (int)pev.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return -1;
            pev.push_back(e);
            pkind.push_back(0);
        }
        cudaEventRecord(pev[pnext], stream);
        pkind[pnext] = kind;
        return pnext;
    }
    void prof_end(int k, long long elements) {
        if (k < 0) return;
        cudaEventRecord(pev[k + 1], stream);
        pnext = k + 2;
        if (pkind[k] == 0) {
            prof_launches += 1;
            prof_elements += elements;
        } else {
            tprof_launches += 1;
        }
    }
    void prof_collect() {
        for (int k = 0; k + 1 < pnext; k += 2) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, pev[k], pev[k + 1]) == cudaSuccess) (pkind[k] == 0 ? prof_ms : tprof_ms) += ms;
        }
        pnext = 0;
    }
};

#define CK(call)                                                                                              \
    do {                                                                                                      \
        cudaError_t e_ = (call);                                                                              \
        if (e_ != cudaSuccess)                                                                                \
            return ctx->fail(OSAM_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

// checked kernel launch, counted
#define LK(call)          \
    do {                  \
        CK(call);         \
        ++ctx->launches;  \
    } while (0)

#define CKA(ptr)                                                                                         \
    do {                                                                                                 \
        if (!(ptr)) return ctx->fail(OSAM_ENOMEM, "device allocation failed (%s:%d)", __FILE__, __LINE__); \
    } while (0)

#define RET(expr)                       \
    do {                                \
        if (int r_ = (expr)) return r_; \
    } while (0)

namespace osam {
namespace host {

inline int upload(osam_ctx* ctx, void* dst, const void* src, size_t bytes) {
    if (bytes == 0) return OSAM_OK;
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, ctx->stream));
    return OSAM_OK;
}

// Address at which the context's kernels can read or write the caller's buffer p in place: device
// memory of the context's device, or page-locked host memory mapped into the device's address space
// (cudaHostAlloc, cudaHostRegister; torch's pinned tensors).  nullptr for anything else (pageable
// host memory, managed memory, another device's memory): those are staged through the scratch buffer
// with a copy.
inline void* direct_view(osam_ctx* ctx, const void* p) {
    cudaPointerAttributes at{};
    if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();   // an unregistered host pointer may leave an error behind on older runtimes
        return nullptr;
    }
    if (at.type == cudaMemoryTypeDevice) return at.device == ctx->device ? at.devicePointer : nullptr;
    if (at.type == cudaMemoryTypeHost) return at.devicePointer;
    return nullptr;
}

// Device-readable form of the caller's n doubles at p: p's own device view when direct_view gives one,
// else the staging buffer, filled by an asynchronous copy in stream order.
inline int stage_in(osam_ctx* ctx, const double* p, size_t n, const double** out) {
    if (const void* d = direct_view(ctx, p)) {
        *out = static_cast<const double*>(d);
        return OSAM_OK;
    }
    RET(upload(ctx, ctx->scratch, p, sizeof(double) * n));
    *out = ctx->scratch;
    return OSAM_OK;
}

template <typename T>
inline int to_host(osam_ctx* ctx, std::vector<T>& out, const T* src, size_t n) {
    out.resize(n);
    if (n == 0) return OSAM_OK;
    CK(cudaMemcpyAsync(out.data(), src, n * sizeof(T), cudaMemcpyDefault, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return OSAM_OK;
}

inline int check_device(osam_ctx* ctx, int device) {
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) return ctx->fail(OSAM_ECUDA, "no CUDA device available (%s)", cudaGetErrorString(e));
    if (device < 0 || device >= n) return ctx->fail(OSAM_EINVAL, "device %d out of range (%d devices)", device, n);
    CK(cudaSetDevice(device));
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, device));
    if (prop.major < 10)
        return ctx->fail(OSAM_ECUDA, "device %d is sm_%d%d; libosam is built for sm_103a", device, prop.major, prop.minor);
    return OSAM_OK;
}

inline bool valid(osam_ctx* ctx, int inst, int sub) {
    return ctx && inst >= 0 && inst < ctx->n_inst && sub >= 0 && sub < (int)ctx->slots.size();
}

// controller.cu: per-step sequences, the implicit intervals, the controller-step graph
bool trace_fuse(osam_ctx* ctx, int s, const double* u, int slot, TraceFuse& tr);
int fom_substep(osam_ctx* ctx, int s, int j, const int* active, long long ne);
int last_trace(osam_ctx* ctx, int s, const int* active);
int any_set(osam_ctx* ctx, const int* mask, int n, bool& any);
int advance_implicit(osam_ctx* ctx, int s, const int* active);
int while_handle(osam_ctx* ctx, cudaStream_t st, cudaGraphConditionalHandle* h);
int while_node(osam_ctx* ctx, cudaStream_t st, cudaGraphConditionalHandle h, cudaGraph_t* body);
int enqueue_implicit_captured(osam_ctx* ctx, int s, const int* active);
int enqueue_implicit(osam_ctx* ctx, int s, const int* active);
int advance_slot(osam_ctx* ctx, int s, const int* active);
bool pipelined_pair(const osam_ctx* ctx, int s);
int advance_pair(osam_ctx* ctx, int s, const int* active);
int transfer_cpl(osam_ctx* ctx, CplH& c, const int* active);
int zoh_cpl(osam_ctx* ctx, CplH& c, const int* active);
int saverest_all(osam_ctx* ctx, const int* active, int restore);
int norms_all(osam_ctx* ctx, const int* active);
int enqueue_begin(osam_ctx* ctx);
int additive_sweep(osam_ctx* ctx, const int* act);
int enqueue_iteration(osam_ctx* ctx, int use_cond);
int build_graph(osam_ctx* ctx);
int read_ctl(osam_ctx* ctx);

// setup.cu: validation, device data of every subdomain group and coupling, the autotuner
int validate_topology(osam_ctx* ctx, int n, const osam_problem_desc* descs);
std::vector<int2> make_blocks(const std::vector<int>& counts, int block, std::vector<int>* first_block);
int set_eblocks(osam_ctx* ctx, FomGroupH& G, int block);
int check_stability(osam_ctx* ctx, FomGroupH& G, int s, int n, const osam_problem_desc* descs);
int set_tiles(osam_ctx* ctx, FomGroupH& G);
int setup_fom_group(osam_ctx* ctx, FomGroupH& G, int s, int n, const osam_problem_desc* descs);
int setup_rom_group(osam_ctx* ctx, RomGroupH& G, int s, int n, const osam_problem_desc* descs);
int setup_couplings(osam_ctx* ctx, int n, const osam_problem_desc* descs,
                    const std::vector<std::vector<std::vector<uint8_t>>>& masks);
int setup_controller(osam_ctx* ctx);
int select_instance(osam_ctx* ctx, int inst);
int initial_accel(osam_ctx* ctx, const int* mask);
int autotune(osam_ctx* ctx);
int init_impl(osam_ctx* ctx, int n, const osam_problem_desc* descs);

}  // namespace host
}  // namespace osam
