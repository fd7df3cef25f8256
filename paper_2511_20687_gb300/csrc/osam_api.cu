// Host runtime of libosam: context construction for one problem or a batch of instances
// (schwarz_init / osam_batch_init), the O-SAM controller (Algorithm 1 of the paper with the
// criterion of Eq. conv_criterion) as a CUDA graph whose Schwarz iterations run in a while node, or
// as a host-driven loop, state I/O, the element-level operators and the adjoint rollout.  Every
// numerical step runs in the kernels of step_kernels.cu, fom_kernels.cu, rom_kernels.cu and
// adjoint_kernels.cu; this file only allocates, sequences and checks.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "osam.h"
#include "osam_internal.h"

using namespace osam;

namespace {

thread_local std::string g_init_error;

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

}  // namespace

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
void set_thread_error(const std::string& msg) { g_init_error = msg; }
}  // namespace osam

namespace {

int upload(osam_ctx* ctx, void* dst, const void* src, size_t bytes) {
    if (bytes == 0) return OSAM_OK;
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, ctx->stream));
    return OSAM_OK;
}

template <typename T>
int to_host(osam_ctx* ctx, std::vector<T>& out, const T* src, size_t n) {
    out.resize(n);
    if (n == 0) return OSAM_OK;
    CK(cudaMemcpyAsync(out.data(), src, n * sizeof(T), cudaMemcpyDefault, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return OSAM_OK;
}

int check_device(osam_ctx* ctx, int device) {
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

// ------------------------------------------------------------------------------------------------
// per-step sequences (used by the graph capture and by the host-driven loop)
// ------------------------------------------------------------------------------------------------
// traces of the couplings fed by FOM slot s at history slot `slot` (state u^slot in buffer u)
bool trace_fuse(osam_ctx* ctx, int s, const double* u, int slot, TraceFuse& tr) {
    tr = TraceFuse{};
    for (CplH& c : ctx->cpls) {
        if (c.src != s) continue;
        if (tr.n == kMaxFusedTraces) return false;
        tr.c[tr.n++] = c.d;
    }
    tr.u = u;
    tr.slot = slot;
    return true;
}

// substep j + 1 of FOM slot s: internal force at u^{j+1} (with the trace of substep j folded into the
// same launch), corrector of j + 1 and predictor of j + 2
int fom_substep(osam_ctx* ctx, int s, int j, const int* active, long long ne) {
    const Slot& S = ctx->slots[s];
    FomB& g = ctx->slots[s].fom.d;
    double* X = g.u[(j + 1) & 1];
    double* Y = g.u[j & 1];
    TraceFuse tr;
    const bool fuse = j > 0 && trace_fuse(ctx, s, g.u[j & 1], j, tr);
    if (j > 0 && !fuse)
        for (CplH& c : ctx->cpls)
            if (c.src == s) LK(launch_trace_b(c.d, active, g, g.u[j & 1], j, ctx->stream));
    const int pk = ctx->prof_begin();
    LK(launch_force_b(g, active, ctx->scatter, ctx->stream, fuse ? &tr : nullptr));
    ctx->prof_end(pk, ne);
    LK(launch_node_b(g, active, ctx->scatter, j + 1, (j + 2 <= S.nsub) ? j + 2 : -1, 0, X, Y, S.dt, ctx->stream));
    return OSAM_OK;
}

// trace of the last substep of FOM slot s (no force launch follows it within the interval)
int last_trace(osam_ctx* ctx, int s, const int* active) {
    FomB& g = ctx->slots[s].fom.d;
    const int n = ctx->slots[s].nsub;
    for (CplH& c : ctx->cpls)
        if (c.src == s) LK(launch_trace_b(c.d, active, g, g.u[n & 1], n, ctx->stream));
    return OSAM_OK;
}

// any instance of a per-instance mask still set (synchronises the stream)
int any_set(osam_ctx* ctx, const int* mask, int n, bool& any) {
    CK(cudaMemcpyAsync(ctx->imp_h, mask, sizeof(int) * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    any = false;
    for (int i = 0; i < n; ++i) any |= ctx->imp_h[i] == 1;
    return OSAM_OK;
}

constexpr int kNewtonMax = 25;         // Newton iterations per substep
constexpr double kNewtonTol2 = 1e-24;  // |R|^2 <= kNewtonTol2 |R(u~)|^2
constexpr double kNewtonInc2 = 1e-28;  // or an increment |du|^2 <= kNewtonInc2 |u|^2 (rounding level of u)
constexpr int kCgMax = 1000;           // CG iterations per Newton step
constexpr int kCgCheck = 8;            // CG iterations between host checks of the activity mask
constexpr double kCgTol2 = 1e-26;      // floor of the CG test r.z <= eta^2 (r.z)_0 (eta: the Newton forcing term)

// Implicit Newmark interval of FOM slot s (beta = 1/4, gamma = 1/2): per substep the predictor, a
// Newton solve of M (u - u~) c0 + f_int(u) = 0 (c0 = 1 / (beta dt^2)) with mass-preconditioned
// conjugate gradients on the exact tangent, until |R| <= 1e-12 |R(u~)| or an increment at the rounding
// level of u (at most 25 Newton steps), the corrector and the traces of the new level.  Each CG solve
// is inexact (Eisenstat-Walker forcing term: relative tolerance min(1e-6, (|R_k| / |R_k-1|)^2), floor
// 1e-13), so early Newton steps do not over-solve; the Newton test itself is unchanged.
// Activity is tracked per instance on the device: Newton (nact: 1 iterating, 0 converged, 2 failed)
// and CG (cgact); the host reads the masks to end the loops.
int advance_implicit(osam_ctx* ctx, int s, const int* active) {
    FomB& g = ctx->slots[s].fom.d;
    const int n = g.n_inst;
    const double dt = ctx->slots[s].dt, c0 = 4.0 / (dt * dt);
    for (int j = 0; j < ctx->slots[s].nsub; ++j) {
        LK(launch_imp_predict_b(g, active, j + 1, dt, ctx->stream));
        LK(launch_mask_copy(n, active, g.nact, ctx->stream));
        LK(launch_mask_copy(n, active, g.cgact, ctx->stream));
        for (int it = 0; it < kNewtonMax; ++it) {
            if (g.lin) LK(launch_force_lin_b(g, g.nact, ctx->stream));
            else LK(launch_force_b(g, g.nact, kGather, ctx->stream, nullptr));
            LK(launch_imp_residual_b(g, g.nact, c0, ctx->stream));
            LK(launch_imp_reduce_b(g, g.nact, 0, it == 0, kNewtonTol2, ctx->stream));
            bool any = false;
            RET(any_set(ctx, g.nact, n, any));
            if (!any) break;
            for (int k = 0; k < kCgMax;) {
                for (int q = 0; q < kCgCheck; ++q, ++k) {
                    const int pk = ctx->prof_begin(1);
                    if (g.lin) LK(launch_tangent_lin_b(g, g.cgact, ctx->stream));
                    else LK(launch_tangent_b(g, g.cgact, ctx->stream));
                    ctx->prof_end(pk, 0);
                    LK(launch_cg_ap_b(g, g.cgact, c0, ctx->stream));
                    LK(launch_cg_step_b(g, g.cgact, c0, kCgTol2, ctx->stream));
                    LK(launch_cg_dir_b(g, g.cgact, c0, ctx->stream));
                }
                bool cg = false;
                RET(any_set(ctx, g.cgact, n, cg));
                if (!cg) break;
            }
            LK(launch_imp_update_b(g, g.nact, ctx->stream));
            LK(launch_imp_reduce_b(g, g.nact, 3, 0, kNewtonInc2, ctx->stream));
        }
        LK(launch_imp_finish_b(g, active, j + 1, dt, c0, ctx->stream));
        for (CplH& c : ctx->cpls)
            if (c.src == s) LK(launch_trace_b(c.d, active, g, g.u[0], j + 1, ctx->stream));
    }
    return OSAM_OK;
}

// ---- implicit interval as a graph with device-side loops ------------------------------------------
// A conditional WHILE node added to the graph being captured on stream st (the handle must exist
// before the kernel that sets its entry value is captured, so it is created first).
int while_handle(osam_ctx* ctx, cudaStream_t st, cudaGraphConditionalHandle* h) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    CK(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, nullptr, nullptr, nullptr));
    if (cs != cudaStreamCaptureStatusActive) return ctx->fail(OSAM_ECUDA, "implicit loop outside a capture");
    CK(cudaGraphConditionalHandleCreate(h, g, 0, 0));
    return OSAM_OK;
}

int while_node(osam_ctx* ctx, cudaStream_t st, cudaGraphConditionalHandle h, cudaGraph_t* body) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* ed = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, &ed, &nd));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g, deps, ed, nd, &cp));
    CK(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    *body = cp.conditional.phGraph_out[0];
    return OSAM_OK;
}

// One implicit interval of FOM slot s into the graph being captured on ctx->stream: per substep the
// predictor, a WHILE node over Newton steps whose body holds the residual, a nested WHILE node over
// CG iterations and the update, then the corrector and the traces.  Same kernels and per-instance
// masks as advance_implicit, without host round trips and without masked trailing CG passes.
int enqueue_implicit_captured(osam_ctx* ctx, int s, const int* active) {
    FomB& g = ctx->slots[s].fom.d;
    const int n = g.n_inst;
    const double dt = ctx->slots[s].dt, c0 = 4.0 / (dt * dt);
    cudaStream_t main = ctx->stream;
    for (int j = 0; j < ctx->slots[s].nsub; ++j) {
        LK(launch_imp_predict_b(g, active, j + 1, dt, main));
        LK(launch_mask_copy(n, active, g.nact, main));
        LK(launch_mask_copy(n, active, g.cgact, main));
        cudaGraphConditionalHandle hn, hc;
        cudaGraph_t nbody, cbody;
        RET(while_handle(ctx, main, &hn));
        LK(launch_imp_loop_entry(g, hn, 0, main));
        RET(while_node(ctx, main, hn, &nbody));
        // Newton body on cap[0]
        CK(cudaStreamBeginCaptureToGraph(ctx->cap[0], nbody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        int rc = OSAM_OK;
        {
            cudaStream_t a = ctx->cap[0];
            auto body = [&]() -> int {
                if (g.lin) LK(launch_force_lin_b(g, g.nact, a));
                else LK(launch_force_b(g, g.nact, kGather, a, nullptr));
                LK(launch_imp_residual_b(g, g.nact, c0, a));
                LK(launch_imp_reduce_b(g, g.nact, 0, -1, kNewtonTol2, a));
                RET(while_handle(ctx, a, &hc));
                LK(launch_imp_loop_entry(g, hc, 1, a));
                RET(while_node(ctx, a, hc, &cbody));
                // CG body on cap[1]
                CK(cudaStreamBeginCaptureToGraph(ctx->cap[1], cbody, nullptr, nullptr, 0,
                                                 cudaStreamCaptureModeThreadLocal));
                cudaStream_t b = ctx->cap[1];
                int rc2 = OSAM_OK;
                auto cg = [&]() -> int {
                    if (g.lin) LK(launch_tangent_lin_b(g, g.cgact, b));
                    else LK(launch_tangent_b(g, g.cgact, b));
                    LK(launch_cg_ap_b(g, g.cgact, c0, b));
                    LK(launch_cg_step_b(g, g.cgact, c0, kCgTol2, b));
                    LK(launch_cg_dir_b(g, g.cgact, c0, b));
                    LK(launch_imp_loop_cond(g, hc, 1, kCgMax, b));
                    return OSAM_OK;
                };
                rc2 = cg();
                cudaGraph_t cb = nullptr;
                cudaError_t ec = cudaStreamEndCapture(b, &cb);
                if (rc2) return rc2;
                CK(ec);
                LK(launch_imp_update_b(g, g.nact, a));
                LK(launch_imp_reduce_b(g, g.nact, 3, 0, kNewtonInc2, a));
                LK(launch_imp_loop_cond(g, hn, 0, kNewtonMax, a));
                return OSAM_OK;
            };
            rc = body();
        }
        cudaGraph_t nb = nullptr;
        cudaError_t ec = cudaStreamEndCapture(ctx->cap[0], &nb);
        if (rc) return rc;
        CK(ec);
        LK(launch_imp_finish_b(g, active, j + 1, dt, c0, main));
        for (CplH& c : ctx->cpls)
            if (c.src == s) LK(launch_trace_b(c.d, active, g, g.u[0], j + 1, main));
    }
    return OSAM_OK;
}

// implicit interval of FOM slot s: inside a controller-step capture its nodes join that graph;
// otherwise an instantiated graph of the interval (built once per activity mask) is launched; with
// kernel-level profiling on, the host-driven loop (CUDA events around every tangent launch)
int enqueue_implicit(osam_ctx* ctx, int s, const int* active) {
    cudaStreamCaptureStatus cs;
    CK(cudaStreamIsCapturing(ctx->stream, &cs));
    if (cs == cudaStreamCaptureStatusActive) return enqueue_implicit_captured(ctx, s, active);
    if (ctx->prof) return advance_implicit(ctx, s, active);
    for (osam_ctx::ImpExec& x : ctx->imp_exec)
        if (x.slot == s && x.active == active) {
            CK(cudaGraphLaunch(x.exec, ctx->stream));
            ctx->launches += x.kernels;
            return OSAM_OK;
        }
    if (!ctx->cap[0])
        for (cudaStream_t& c : ctx->cap) CK(cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking));
    const long long l0 = ctx->launches;
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_implicit_captured(ctx, s, active);
    cudaError_t ec = cudaStreamEndCapture(ctx->stream, &graph);
    const long long nk = ctx->launches - l0;
    ctx->launches = l0;
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    CK(ec);
    cudaGraphExec_t exec = nullptr;
    CK(cudaGraphInstantiate(&exec, graph, 0));
    ctx->imp_exec.push_back({s, active, graph, exec, nk});
    CK(cudaGraphLaunch(exec, ctx->stream));
    ctx->launches += nk;
    return OSAM_OK;
}

int advance_slot(osam_ctx* ctx, int s, const int* active) {
    Slot& S = ctx->slots[s];
    if (S.kind == OSAM_FOM && S.fom.d.implicit) return enqueue_implicit(ctx, s, active);
    if (S.kind == OSAM_FOM) {
        FomB& g = S.fom.d;
        long long ne = 0;
        for (const InstFom& I : S.fom.inst) ne += I.ne;
        LK(launch_node_b(g, active, ctx->scatter, -1, 1, 1, g.u[0], g.u[1], S.dt, ctx->stream));
        for (int j = 0; j < S.nsub; ++j) RET(fom_substep(ctx, s, j, active, ne));
        RET(last_trace(ctx, s, active));
        if (S.nsub & 1) LK(launch_copy_u10_b(g, active, ctx->stream));
    } else {
        RomB& r = S.rom.d;
        LK(launch_rom_record0_b(r, active, ctx->stream));
        LK(launch_rom_project_b(r, active, 1, S.nsub, ctx->stream));
        for (int j = 0; j < S.nsub; ++j) LK(launch_rom_step_b(r, active, j + 1, S.dt, 0, ctx->stream));
    }
    return OSAM_OK;
}

// FOM slot s followed by ROM slot s + 1 whose only source among the slots before it is s: the ROM's
// substep j needs only the FOM's trace of substep j, so it can run one substep behind the FOM.
bool pipelined_pair(const osam_ctx* ctx, int s) {
    if (s + 1 >= (int)ctx->slots.size()) return false;
    if (ctx->slots[s].kind != OSAM_FOM || ctx->slots[s + 1].kind != OSAM_ROM) return false;
    if (ctx->slots[s].fom.d.implicit) return false;
    if (ctx->slots[s].nsub != ctx->slots[s + 1].nsub) return false;  // substep j <-> j needs equal levels
    bool fed = false;
    for (const CplH& c : ctx->cpls) {
        if (c.dst != s + 1 || c.src > s) continue;
        if (c.src != s) return false;
        fed = true;
    }
    return fed;
}

// FOM slot s on the main stream and ROM slot s + 1 on the side stream, one substep behind: after the
// FOM's trace of substep j the side stream publishes that slot of every coupling s -> s + 1, projects
// it onto the ROM's boundary basis and takes the ROM's substep j.  The same kernels in the same
// per-subdomain order as advance_slot(s), transfer(s -> s + 1), advance_slot(s + 1), so the results
// are identical; only the two subdomains' work overlaps.
int advance_pair(osam_ctx* ctx, int s, const int* active) {
    const int nsub = ctx->slots[s].nsub;
    const double dt = ctx->slots[s].dt;
    FomB& g = ctx->slots[s].fom.d;
    RomB& r = ctx->slots[s + 1].rom.d;
    long long ne = 0;
    for (const InstFom& I : ctx->slots[s].fom.inst) ne += I.ne;
    CK(cudaEventRecord(ctx->ev_fork, ctx->stream));
    CK(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
    LK(launch_rom_record0_b(r, active, ctx->side));
    LK(launch_node_b(g, active, ctx->scatter, -1, 1, 1, g.u[0], g.u[1], dt, ctx->stream));
    // the trace of substep j is complete after the force launch of substep j + 1 (or the last trace)
    auto rom_substep = [&](int j) -> int {
        CK(cudaEventRecord(ctx->ev_fork, ctx->stream));
        CK(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
        for (CplH& c : ctx->cpls)
            if (c.src == s && c.dst == s + 1) LK(launch_publish_b(c.d, active, j, 1, nsub, nsub, ctx->side));
        LK(launch_rom_project_b(r, active, j, j, ctx->side));
        LK(launch_rom_step_b(r, active, j, dt, 0, ctx->side));
        return OSAM_OK;
    };
    for (int j = 0; j < nsub; ++j) {
        RET(fom_substep(ctx, s, j, active, ne));
        if (j > 0) RET(rom_substep(j));
    }
    RET(last_trace(ctx, s, active));
    RET(rom_substep(nsub));
    if (nsub & 1) LK(launch_copy_u10_b(g, active, ctx->stream));
    CK(cudaEventRecord(ctx->ev_join, ctx->side));
    CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0));
    return OSAM_OK;
}

// src's interval trace onto dst's time levels 1..n_dst (temporal interpolant Xi, Sec. 4.1: linear
// between the src levels that bracket each dst level; identity for equal substep counts)
int transfer_cpl(osam_ctx* ctx, CplH& c, const int* active) {
    Slot& src = ctx->slots[c.src];
    const int ns = src.nsub, nd = ctx->slots[c.dst].nsub;
    if (src.kind == OSAM_FOM) LK(launch_publish_b(c.d, active, 1, nd, ns, nd, ctx->stream));
    else LK(launch_rom_reconstruct_b(c.d, active, src.rom.d, 0, ns, nd, ctx->stream));
    return OSAM_OK;
}

// zero-order hold of src's current state into every dst level (and the FOM trace's level 0)
int zoh_cpl(osam_ctx* ctx, CplH& c, const int* active) {
    Slot& src = ctx->slots[c.src];
    const int ns = src.nsub, nd = ctx->slots[c.dst].nsub;
    if (src.kind == OSAM_FOM) LK(launch_zoh_fom_b(c.d, active, src.fom.d, nd, ctx->stream));
    else LK(launch_rom_reconstruct_b(c.d, active, src.rom.d, 1, ns, nd, ctx->stream));
    return OSAM_OK;
}

int saverest_all(osam_ctx* ctx, const int* active, int restore) {
    for (Slot& S : ctx->slots) {
        if (S.kind == OSAM_FOM) LK(launch_saverest_fom_b(S.fom.d, active, restore, ctx->stream));
        else LK(launch_saverest_rom_b(S.rom.d, active, restore, ctx->stream));
    }
    return OSAM_OK;
}

int norms_all(osam_ctx* ctx, const int* active) {
    for (Slot& S : ctx->slots) {
        if (S.kind == OSAM_FOM) LK(launch_norms_fom_b(S.fom.d, active, S.dt, ctx->stream));
        else LK(launch_rom_norms_b(S.rom.d, active, S.dt, ctx->stream));
    }
    return OSAM_OK;
}

// start of a controller step: save the state at t_{k-1}, zero-order hold of every source, flags
int enqueue_begin(osam_ctx* ctx) {
    RET(saverest_all(ctx, nullptr, 0));
    for (CplH& c : ctx->cpls) RET(zoh_cpl(ctx, c, nullptr));
    LK(launch_reset_ctl(ctx->ctl, ctx->stream));
    return OSAM_OK;
}

// additive sweep (Remark additive_sam): every subdomain advances from the boundary data of the previous
// iteration, concurrently on its own stream (subdomain 0 on the context stream); the transfers follow
// the join.  Implicit subdomains synchronise with the host inside their Newton loops, so they are
// enqueued after the explicit ones, whose work is then already in flight.
int additive_sweep(osam_ctx* ctx, const int* act) {
    const int n = (int)ctx->slots.size();
    CK(cudaEventRecord(ctx->ev_fork, ctx->stream));
    cudaStream_t main = ctx->stream;
    int rc = OSAM_OK;
    for (int pass = 0; pass < 2 && rc == OSAM_OK; ++pass)
        for (int s = 0; s < n && rc == OSAM_OK; ++s) {
            const Slot& S = ctx->slots[s];
            const bool imp = S.kind == OSAM_FOM && S.fom.d.implicit;
            if (imp != (pass == 1)) continue;
            if (s > 0) {
                cudaStream_t lane = ctx->lanes[s - 1];
                CK(cudaStreamWaitEvent(lane, ctx->ev_fork, 0));
                ctx->stream = lane;
            }
            rc = advance_slot(ctx, s, act);
            ctx->stream = main;
            if (rc == OSAM_OK && s > 0) CK(cudaEventRecord(ctx->lane_join[s - 1], ctx->lanes[s - 1]));
        }
    if (rc) return rc;
    for (int s = 1; s < n; ++s) CK(cudaStreamWaitEvent(ctx->stream, ctx->lane_join[s - 1], 0));
    for (CplH& c : ctx->cpls) RET(transfer_cpl(ctx, c, act));
    return OSAM_OK;
}

// one Schwarz iteration for every instance still iterating; instances that continue are restored
// to the saved state for the next iteration
int enqueue_iteration(osam_ctx* ctx, int use_cond) {
    const int* act = ctx->ctl.active;
    if (ctx->additive) {
        RET(additive_sweep(ctx, act));
        RET(norms_all(ctx, act));
        LK(launch_controller(ctx->ctl, ctx->cond, use_cond, ctx->stream));
        RET(saverest_all(ctx, act, 1));
        return OSAM_OK;
    }
    for (int s = 0; s < (int)ctx->slots.size(); ++s) {
        if (pipelined_pair(ctx, s)) {
            RET(advance_pair(ctx, s, act));
            for (CplH& c : ctx->cpls)
                if (c.src == s && c.dst != s + 1) RET(transfer_cpl(ctx, c, act));
            ++s;
        } else {
            RET(advance_slot(ctx, s, act));
        }
        for (CplH& c : ctx->cpls)
            if (c.src == s) RET(transfer_cpl(ctx, c, act));
    }
    RET(norms_all(ctx, act));
    LK(launch_controller(ctx->ctl, ctx->cond, use_cond, ctx->stream));
    RET(saverest_all(ctx, act, 1));
    return OSAM_OK;
}

int build_graph(osam_ctx* ctx) {
    if (ctx->exec) return OSAM_OK;
    const long long launches0 = ctx->launches;
    CK(cudaGraphCreate(&ctx->graph, 0));
    CK(cudaGraphConditionalHandleCreate(&ctx->cond, ctx->graph, 1, cudaGraphCondAssignDefault));
    CK(cudaStreamBeginCaptureToGraph(ctx->stream, ctx->graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_begin(ctx);
    ctx->graph_begin_launches = ctx->launches - launches0;
    cudaGraph_t g = nullptr;
    cudaError_t ec = cudaStreamEndCapture(ctx->stream, &g);
    if (rc) return rc;
    CK(ec);
    // the while node depends on every leaf of the begin nodes
    size_t n = 0;
    CK(cudaGraphGetNodes(ctx->graph, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n), leaves;
    CK(cudaGraphGetNodes(ctx->graph, nodes.data(), &n));
    for (cudaGraphNode_t nd : nodes) {
        size_t nd_out = 0;
        CK(cudaGraphNodeGetDependentNodes(nd, nullptr, nullptr, &nd_out));
        if (nd_out == 0) leaves.push_back(nd);
    }
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = ctx->cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode;
    CK(cudaGraphAddNode(&wnode, ctx->graph, leaves.data(), nullptr, leaves.size(), &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(ctx->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const long long body0 = ctx->launches;
    rc = enqueue_iteration(ctx, 1);
    ctx->graph_body_launches = ctx->launches - body0;
    ec = cudaStreamEndCapture(ctx->stream, &body);
    if (rc) return rc;
    CK(ec);
    CK(cudaGraphInstantiate(&ctx->exec, ctx->graph, cudaGraphInstantiateFlagUseNodePriority));
    ctx->launches = launches0;  // capture issued nothing
    return OSAM_OK;
}

int read_ctl(osam_ctx* ctx) {
    const int n = ctx->n_inst;
    CK(cudaMemcpyAsync(ctx->iters_h, ctx->ctl.iters, sizeof(int) * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ctx->status_h, ctx->ctl.status, sizeof(int) * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ctx->cnum_h, ctx->ctl.cnum, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ctx->cden_h, ctx->ctl.cden, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
    return OSAM_OK;
}

// kernels one Schwarz iteration launches (for the launch count of the graph path)
// ------------------------------------------------------------------------------------------------
// set-up
// ------------------------------------------------------------------------------------------------
int validate_topology(osam_ctx* ctx, int n, const osam_problem_desc* descs) {
    const osam_problem_desc& d0 = descs[0];
    if (d0.n_subdomains < 1 || d0.n_subdomains > kMaxSlots || !d0.subdomains)
        return ctx->fail(OSAM_EINVAL, "1..%d subdomains required", kMaxSlots);
    if (d0.n_couplings < 0 || (d0.n_couplings > 0 && !d0.couplings)) return ctx->fail(OSAM_EINVAL, "bad couplings");
    if (!(d0.dt > 0.0) || d0.n_substeps < 1 || d0.max_iters < 1)
        return ctx->fail(OSAM_EINVAL, "dt, n_substeps and max_iters must be positive");
    if (d0.precision != OSAM_FP64 && d0.precision != OSAM_FP32_FORCE && d0.precision != OSAM_F32X2_FORCE)
        return ctx->fail(OSAM_EINVAL, "bad precision");
    if (d0.scatter < OSAM_SCATTER_AUTO || d0.scatter > OSAM_SCATTER_GATHER_TILED)
        return ctx->fail(OSAM_EINVAL, "bad scatter mode");
    if (d0.schwarz != OSAM_MULTIPLICATIVE && d0.schwarz != OSAM_ADDITIVE)
        return ctx->fail(OSAM_EINVAL, "bad Schwarz variant");
    for (int k = 0; k < d0.n_couplings; ++k) {
        const osam_coupling_desc& c = d0.couplings[k];
        if (c.dst < 0 || c.dst >= d0.n_subdomains || c.src < 0 || c.src >= d0.n_subdomains || c.dst == c.src)
            return ctx->fail(OSAM_EINVAL, "coupling %d: bad indices", k);
    }
    for (int i = 0; i < n; ++i) {
        const osam_problem_desc& d = descs[i];
        if (d.n_subdomains != d0.n_subdomains || d.n_couplings != d0.n_couplings || d.dt != d0.dt ||
            d.n_substeps != d0.n_substeps || d.max_iters != d0.max_iters || d.tol_abs != d0.tol_abs ||
            d.tol_rel != d0.tol_rel || d.precision != d0.precision || d.device != d0.device || !d.subdomains ||
            d.schwarz != d0.schwarz)
            return ctx->fail(OSAM_EINVAL, "instance %d: controller settings differ from instance 0", i);
        for (int s = 0; s < d0.n_subdomains; ++s) {
            const osam_subdomain_desc& a = d.subdomains[s];
            const osam_subdomain_desc& b = d0.subdomains[s];
            if (a.kind != OSAM_FOM && a.kind != OSAM_ROM) return ctx->fail(OSAM_EINVAL, "subdomain %d: bad kind", s);
            if (a.kind != b.kind || (a.kind == OSAM_FOM && a.material != b.material))
                return ctx->fail(OSAM_EINVAL, "instance %d subdomain %d: kind / material differ from instance 0", i, s);
            if (a.nx < 1 || a.ny < 1 || a.nz < 1 || !(a.h > 0.0))
                return ctx->fail(OSAM_EINVAL, "instance %d subdomain %d: bad mesh", i, s);
            if ((long long)(a.nx + 1) * (a.ny + 1) * (a.nz + 1) > (1LL << 30))
                return ctx->fail(OSAM_EINVAL, "instance %d subdomain %d too large", i, s);
            if (!a.u0) return ctx->fail(OSAM_EINVAL, "instance %d subdomain %d: u0 required", i, s);
            if (a.kind == OSAM_FOM && a.material != OSAM_LINEAR_ELASTIC && a.material != OSAM_NEO_HOOKEAN &&
                a.material != OSAM_SAINT_VENANT_KIRCHHOFF)
                return ctx->fail(OSAM_EINVAL, "subdomain %d: bad material", s);
            if (a.kind == OSAM_FOM && !(a.rho > 0.0))
                return ctx->fail(OSAM_EINVAL, "instance %d subdomain %d: rho must be positive", i, s);
            if (a.kind == OSAM_FOM && a.integrator != OSAM_EXPLICIT && a.integrator != OSAM_IMPLICIT)
                return ctx->fail(OSAM_EINVAL, "instance %d subdomain %d: bad integrator", i, s);
            if (a.n_substeps < 0 || a.n_substeps > (1 << 20) || a.n_substeps != b.n_substeps)
                return ctx->fail(OSAM_EINVAL, "instance %d subdomain %d: bad or differing n_substeps", i, s);
            if (a.kind == OSAM_FOM && a.integrator != b.integrator)
                return ctx->fail(OSAM_EINVAL, "instance %d subdomain %d: integrator differs from instance 0", i, s);
            if (a.kind == OSAM_FOM && a.integrator == OSAM_IMPLICIT && d0.precision != OSAM_FP64)
                return ctx->fail(OSAM_EINVAL, "subdomain %d: implicit integration needs OSAM_FP64", s);
        }
        for (int k = 0; k < d0.n_couplings; ++k) {
            if (!d.couplings || d.couplings[k].dst != d0.couplings[k].dst || d.couplings[k].src != d0.couplings[k].src ||
                !d.couplings[k].nodes)
                return ctx->fail(OSAM_EINVAL, "instance %d coupling %d differs from instance 0", i, k);
        }
    }
    return OSAM_OK;
}

std::vector<int2> make_blocks(const std::vector<int>& counts, int block, std::vector<int>* first_block) {
    std::vector<int2> out;
    if (first_block) first_block->assign(counts.size() + 1, 0);
    for (size_t i = 0; i < counts.size(); ++i) {
        if (first_block) (*first_block)[i] = (int)out.size();
        for (int b = 0; b < counts[i]; b += block) out.push_back(make_int2((int)i, b));
    }
    if (first_block) (*first_block)[counts.size()] = (int)out.size();
    return out;
}

int set_eblocks(osam_ctx* ctx, FomGroupH& G, int block) {
    std::vector<int> ne;
    for (const InstFom& I : G.inst) ne.push_back(I.ne);
    std::vector<int2> eb = make_blocks(ne, block, nullptr);
    int2* d = ctx->alloc<int2>(eb.size());
    CKA(d);
    RET(upload(ctx, d, eb.data(), sizeof(int2) * eb.size()));
    G.d.eblk = d;
    G.d.n_eblk = (int)eb.size();
    G.d.eblock = block;
    return OSAM_OK;
}

// Explicit stability of every instance of FOM slot s: dt <= h sqrt(rho / max_e max(3 lambda_e + 2 mu_e,
// 2 mu_e)) (element eigenvalue bound of the lumped-mass system at the reference configuration; the
// Neo-Hookean law linearises to the same lambda, mu).  A relative allowance of 1e-9 keeps a step that
// sits exactly on the limit.
int check_stability(osam_ctx* ctx, FomGroupH& G, int s, int n, const osam_problem_desc* descs) {
    unsigned long long* mod = ctx->alloc<unsigned long long>(n);
    int* bad = ctx->alloc<int>(1);
    CKA(mod); CKA(bad);
    CK(cudaMemsetAsync(mod, 0, sizeof(unsigned long long) * n, ctx->stream));
    CK(cudaMemsetAsync(bad, 0, sizeof(int), ctx->stream));
    CK(launch_cfl_modulus(G.d, mod, bad, ctx->stream));
    std::vector<unsigned long long> mh;
    std::vector<int> bh;
    RET(to_host(ctx, mh, mod, n));
    RET(to_host(ctx, bh, bad, 1));
    if (bh[0]) return ctx->fail(OSAM_EINVAL, "subdomain %d: material not positive definite (mu > 0 and "
                                             "3 lambda + 2 mu > 0 required)", s);
    for (int i = 0; i < n; ++i) {
        double m;
        std::memcpy(&m, &mh[i], sizeof(double));
        const double lim = G.grid[i].h * std::sqrt(descs[i].subdomains[s].rho / m);
        const double dt = ctx->slots[s].dt;
        if (!G.d.implicit && dt > lim * (1.0 + 1e-9))
            return ctx->fail(OSAM_ECFL, "instance %d subdomain %d: dt = %.6e above the explicit stability limit "
                                        "%.6e", i, s, dt, lim);
    }
    return OSAM_OK;
}

// 8x4x4 element tiles of every instance of a FOM group (the tiled force kernel's blocks)
int set_tiles(osam_ctx* ctx, FomGroupH& G) {
    std::vector<int4> tb;
    for (int i = 0; i < (int)G.inst.size(); ++i) {
        const InstFom& I = G.inst[i];
        for (int k0 = 0; k0 < I.nz; k0 += 4)
            for (int j0 = 0; j0 < I.ny; j0 += 4)
                for (int i0 = 0; i0 < I.nx; i0 += 8) tb.push_back(make_int4(i, i0, j0, k0));
    }
    int4* d = ctx->alloc<int4>(tb.size());
    CKA(d);
    RET(upload(ctx, d, tb.data(), sizeof(int4) * tb.size()));
    G.d.tblk = d;
    G.d.n_tblk = (int)tb.size();
    return OSAM_OK;
}

int setup_fom_group(osam_ctx* ctx, FomGroupH& G, int s, int n, const osam_problem_desc* descs) {
    const bool fp32 = ctx->precision == OSAM_FP32_FORCE;
    long long NN = 0, NE = 0, H = 0;
    G.inst.resize(n);
    for (int i = 0; i < n; ++i) {
        const Grid& g = G.grid[i];
        const osam_subdomain_desc& d = descs[i].subdomains[s];
        InstFom& I = G.inst[i];
        I = InstFom{};
        I.nx = g.nx; I.ny = g.ny; I.nz = g.nz; I.nn = g.nn(); I.ne = g.ne(); I.ns = G.ns[i];
        I.invh = 1.0 / g.h;
        I.w8 = g.h * g.h / 8.0;
        I.lam = d.lambda; I.mu = d.mu;
        I.node_off = NN; I.elem_off = NE; I.hist_off = H;
        NN += I.nn; NE += I.ne; H += (long long)(ctx->slots[s].nsub + 1) * 9 * I.ns;
    }
    FomB& B = G.d;
    B.n_inst = n; B.NN = NN; B.NE = NE;
    B.material = descs[0].subdomains[s].material;
    B.fp32 = fp32;
    B.df32 = ctx->precision == OSAM_F32X2_FORCE;
    B.scatter = ctx->scatter;
    double* minv = ctx->alloc<double>(NN);
    uint8_t* clamp = ctx->alloc<uint8_t>(NN);
    int* srow = ctx->alloc<int>(NN);
    CKA(minv); CKA(clamp); CKA(srow);
    B.minv = minv; B.clamp = clamp; B.srow = srow;
    for (int b = 0; b < 2; ++b) CKA(B.u[b] = ctx->alloc<double>(3 * NN));
    CKA(B.v = ctx->alloc<double>(3 * NN));
    CKA(B.a = ctx->alloc<double>(3 * NN));
    CKA(B.f = ctx->alloc<double>(3 * NN));
    CKA(B.fe = ctx->alloc<double>(24 * NE));  // FP64-sized: the FP64 initial force also uses it
    CKA(B.su = ctx->alloc<double>(3 * NN));
    CKA(B.sv = ctx->alloc<double>(3 * NN));
    CKA(B.sa = ctx->alloc<double>(3 * NN));
    CKA(B.pu = ctx->alloc<double>(3 * NN));
    CKA(B.pv = ctx->alloc<double>(3 * NN));
    CKA(B.hist = ctx->alloc<double>(std::max<long long>(H, 1)));
    CKA(B.us = ctx->alloc<double>(3 * NN));
    if (B.df32) CKA(B.u2 = ctx->alloc<float2>(3 * NN));
    B.implicit = descs[0].subdomains[s].integrator == OSAM_IMPLICIT;
    if (B.implicit) {
        ctx->any_implicit = true;
        CKA(B.ut = ctx->alloc<double>(3 * NN));
        CKA(B.cg_x = ctx->alloc<double>(3 * NN));
        CKA(B.cg_r = ctx->alloc<double>(3 * NN));
        CKA(B.cg_p = ctx->alloc<double>(3 * NN));
        CKA(B.cg_ap = ctx->alloc<double>(3 * NN));
        for (double** p : {&B.rn2, &B.r0, &B.rr, &B.rrn, &B.rr0, &B.pap, &B.cgtol2, &B.alpha, &B.beta})
            CKA(*p = ctx->alloc<double>(n));
        CKA(B.iticket = ctx->alloc<unsigned int>(n));
        CK(cudaMemsetAsync(B.iticket, 0, sizeof(unsigned int) * n, ctx->stream));
        CKA(B.istat = ctx->alloc<long long>(2 * n));
        CKA(B.iloop = ctx->alloc<int>(2));
        if (B.material == OSAM_NEO_HOOKEAN) CKA(B.lin = ctx->alloc<double>((long long)kLinPerGp * 8 * NE));
        CK(cudaMemsetAsync(B.istat, 0, sizeof(long long) * 2 * n, ctx->stream));
        CKA(B.nact = ctx->alloc<int>(n));
        CKA(B.cgact = ctx->alloc<int>(n));
        CK(cudaMemsetAsync(B.nact, 0, sizeof(int) * n, ctx->stream));
        CK(cudaMemsetAsync(B.cgact, 0, sizeof(int) * n, ctx->stream));
    }
    bool any_le = false, any_me = false;
    for (int i = 0; i < n; ++i) {
        any_le |= descs[i].subdomains[s].lambda_e != nullptr;
        any_me |= descs[i].subdomains[s].mu_e != nullptr;
    }
    double* lam_e = any_le ? ctx->alloc<double>(NE) : nullptr;
    double* mu_e = any_me ? ctx->alloc<double>(NE) : nullptr;
    if (any_le) CKA(lam_e);
    if (any_me) CKA(mu_e);
    for (int i = 0; i < n; ++i) {
        const osam_subdomain_desc& d = descs[i].subdomains[s];
        InstFom& I = G.inst[i];
        if (d.lambda_e) {
            RET(upload(ctx, lam_e + I.elem_off, d.lambda_e, sizeof(double) * I.ne));
            I.lam_e = lam_e + I.elem_off;
        }
        if (d.mu_e) {
            RET(upload(ctx, mu_e + I.elem_off, d.mu_e, sizeof(double) * I.ne));
            I.mu_e = mu_e + I.elem_off;
        }
        CK(launch_lumped_minv(G.grid[i], d.rho, minv + I.node_off, ctx->stream));
        RET(upload(ctx, clamp + I.node_off, G.clamp[i].data(), I.nn));
        RET(upload(ctx, srow + I.node_off, G.srow[i].data(), sizeof(int) * I.nn));
        RET(upload(ctx, ctx->scratch, d.u0, sizeof(double) * 3 * I.nn));
        CK(launch_aos_to_soa(ctx->scratch, B.u[0] + I.node_off, I.nn, NN, ctx->stream));
        if (d.v0) {
            CK(cudaStreamSynchronize(ctx->stream));
            RET(upload(ctx, ctx->scratch, d.v0, sizeof(double) * 3 * I.nn));
            CK(launch_aos_to_soa(ctx->scratch, B.v + I.node_off, I.nn, NN, ctx->stream));
        }
        CK(launch_zero_clamped(I.nn, clamp + I.node_off, B.u[0] + I.node_off, B.v + I.node_off, NN, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));  // the staging buffers are reused by the next instance
    }
    CKA(G.inst_d = ctx->alloc<InstFom>(n));
    RET(upload(ctx, G.inst_d, G.inst.data(), sizeof(InstFom) * n));
    B.inst = G.inst_d;
    std::vector<int> nn;
    for (const InstFom& I : G.inst) nn.push_back(I.nn);
    G.nblk = make_blocks(nn, kNodeBlock, &G.nblk_off);
    int2* nb = ctx->alloc<int2>(G.nblk.size());
    int* nbo = ctx->alloc<int>(G.nblk_off.size());
    CKA(nb); CKA(nbo);
    RET(upload(ctx, nb, G.nblk.data(), sizeof(int2) * G.nblk.size()));
    RET(upload(ctx, nbo, G.nblk_off.data(), sizeof(int) * G.nblk_off.size()));
    B.nblk = nb;
    B.n_nblk = (int)G.nblk.size();
    B.nblk_off = nbo;
    CKA(B.partial = ctx->alloc<double>(2LL * B.n_nblk));
    if (B.implicit) CKA(B.ipart = ctx->alloc<double>(2LL * B.n_nblk));
    RET(set_eblocks(ctx, G, 128));
    RET(set_tiles(ctx, G));
    RET(check_stability(ctx, G, s, n, descs));
    if (B.df32) CK(launch_split_u2_b(B, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return OSAM_OK;
}

int setup_rom_group(osam_ctx* ctx, RomGroupH& G, int s, int n, const osam_problem_desc* descs) {
    G.inst.resize(n);
    G.nfree.resize(n);
    long long nn_tot = 0, nfree_tot = 0, O_tot = 0, PS_tot = 0, kij_tot = 0, kijk_tot = 0, q_tot = 0, qrec_tot = 0,
              ghat_tot = 0, hist_tot = 0, part_tot = 0, phi_tot = 0;
    RomB& B = G.d;
    B.n_inst = n;
    B.gx_max = B.gy_max = B.rs_max = B.r_max = 0;
    std::vector<std::vector<int>> free_dof(n), dof_free(n);
    int max_nn = 1;
    for (int i = 0; i < n; ++i) {
        const osam_subdomain_desc& d = descs[i].subdomains[s];
        InstRom& I = G.inst[i];
        I = InstRom{};
        const int nn = G.grid[i].nn();
        max_nn = std::max(max_nn, nn);
        if (d.r < 1 || d.r > 256) return ctx->fail(OSAM_EINVAL, "instance %d: ROM rank r=%d outside [1, 256]", i, d.r);
        if (d.r_s < 0 || (d.r_s > 0 && !d.Phi_S)) return ctx->fail(OSAM_EINVAL, "instance %d: ROM boundary basis missing", i);
        if (!d.Phi || !d.K || !d.H || !d.c || (d.r_s > 0 && !d.B))
            return ctx->fail(OSAM_EINVAL, "instance %d: ROM operator missing", i);
        dof_free[i].assign(3 * nn, -1);
        for (int nd = 0; nd < nn; ++nd)
            for (int c = 0; c < 3; ++c)
                if (!(G.clamp[i][nd] & (1 << c)) && G.srow[i][nd] < 0) {
                    dof_free[i][3 * nd + c] = (int)free_dof[i].size();
                    free_dof[i].push_back(3 * nd + c);
                }
        G.nfree[i] = (int)free_dof[i].size();
        I.r = d.r; I.rs = d.r_s; I.nsdof = 3 * G.ns[i];
        I.nq = I.r * (I.r + 1) / 2;
        if (d.C && d.r > 128) return ctx->fail(OSAM_EINVAL, "instance %d: cubic ROM rank r=%d above 128", i, d.r);
        I.nc = d.C ? I.r * (I.r + 1) * (I.r + 2) / 6 : 0;
        I.d = I.r + I.nq + I.nc + I.rs + 1;
        I.gx = grid_for(I.d, 128);
        I.gy = grid_for(I.r, 8);
        I.O_off = O_tot; O_tot += (long long)I.r * I.d;
        I.PhiSt_off = PS_tot; PS_tot += (long long)I.rs * I.nsdof;
        I.kij_off = kij_tot; kij_tot += I.nq;
        I.kijk_off = kijk_tot; kijk_tot += I.nc;
        I.q_off = q_tot; q_tot += 3LL * I.r;
        const long long nl = ctx->slots[s].nsub + 1;
        I.qrec_off = qrec_tot; qrec_tot += nl * 3 * I.r;
        I.ghat_off = ghat_tot; ghat_tot += nl * std::max(1, I.rs);
        I.hist_off = hist_tot; hist_tot += nl * 3 * std::max(1, I.nsdof);
        I.partial_off = part_tot; part_tot += (long long)I.gx * I.r;
        B.gx_max = std::max(B.gx_max, I.gx);
        B.gy_max = std::max(B.gy_max, I.gy);
        B.rs_max = std::max(B.rs_max, I.rs);
        B.r_max = std::max(B.r_max, I.r);
        nn_tot += nn;
        nfree_tot += G.nfree[i];
        phi_tot += (long long)G.nfree[i] * I.r;
    }
    double* O = ctx->alloc<double>(O_tot);
    double* PhiSt = ctx->alloc<double>(std::max(1LL, PS_tot));
    short2* kij = ctx->alloc<short2>(std::max(1LL, kij_tot));
    short4* kijk = ctx->alloc<short4>(std::max(1LL, kijk_tot));
    CKA(O); CKA(PhiSt); CKA(kij); CKA(kijk);
    CKA(B.q = ctx->alloc<double>(q_tot));
    CKA(B.sq = ctx->alloc<double>(q_tot));
    CKA(B.pq = ctx->alloc<double>(q_tot));
    CKA(B.qrec = ctx->alloc<double>(qrec_tot));
    CKA(B.ghat = ctx->alloc<double>(ghat_tot));
    CKA(B.hist = ctx->alloc<double>(hist_tot));
    CKA(B.partial = ctx->alloc<double>(part_tot));
    CKA(B.counter = ctx->alloc<unsigned int>(n));
    CKA(B.npart = ctx->alloc<double>(2LL * n));
    double* PhiAll = ctx->alloc<double>(std::max(1LL, phi_tot));
    int* fdAll = ctx->alloc<int>(std::max(1LL, nfree_tot));
    int* dfAll = ctx->alloc<int>(3 * nn_tot);
    uint8_t* clAll = ctx->alloc<uint8_t>(nn_tot);
    int* srAll = ctx->alloc<int>(nn_tot);
    double* uv = ctx->alloc<double>(6LL * max_nn);
    CKA(PhiAll); CKA(fdAll); CKA(dfAll); CKA(clAll); CKA(srAll); CKA(uv);
    G.Phi.resize(n); G.free_dof.resize(n); G.dof_free.resize(n); G.clamp_d.resize(n); G.srow_d.resize(n);
    long long po = 0, fo = 0, no = 0;
    for (int i = 0; i < n; ++i) {
        const osam_subdomain_desc& d = descs[i].subdomains[s];
        InstRom& I = G.inst[i];
        const int nn = G.grid[i].nn();
        G.Phi[i] = PhiAll + po;
        G.free_dof[i] = fdAll + fo;
        G.dof_free[i] = dfAll + 3 * no;
        G.clamp_d[i] = clAll + no;
        G.srow_d[i] = srAll + no;
        RET(upload(ctx, G.Phi[i], d.Phi, sizeof(double) * G.nfree[i] * I.r));
        RET(upload(ctx, G.free_dof[i], free_dof[i].data(), sizeof(int) * G.nfree[i]));
        RET(upload(ctx, G.dof_free[i], dof_free[i].data(), sizeof(int) * 3 * nn));
        RET(upload(ctx, G.clamp_d[i], G.clamp[i].data(), nn));
        RET(upload(ctx, G.srow_d[i], G.srow[i].data(), sizeof(int) * nn));
        po += (long long)G.nfree[i] * I.r;
        fo += G.nfree[i];
        no += nn;
        std::vector<double> K, Hh, Ch, Bh, c, Op((size_t)I.r * I.d);
        RET(to_host(ctx, K, d.K, (size_t)I.r * I.r));
        RET(to_host(ctx, Hh, d.H, (size_t)I.r * I.nq));
        if (I.nc) RET(to_host(ctx, Ch, d.C, (size_t)I.r * I.nc));
        if (I.rs) RET(to_host(ctx, Bh, d.B, (size_t)I.r * I.rs));
        RET(to_host(ctx, c, d.c, (size_t)I.r));
        for (int row = 0; row < I.r; ++row) {
            double* o = Op.data() + (size_t)row * I.d;
            std::copy(K.begin() + (size_t)row * I.r, K.begin() + (size_t)(row + 1) * I.r, o);
            std::copy(Hh.begin() + (size_t)row * I.nq, Hh.begin() + (size_t)(row + 1) * I.nq, o + I.r);
            if (I.nc)
                std::copy(Ch.begin() + (size_t)row * I.nc, Ch.begin() + (size_t)(row + 1) * I.nc, o + I.r + I.nq);
            if (I.rs)
                std::copy(Bh.begin() + (size_t)row * I.rs, Bh.begin() + (size_t)(row + 1) * I.rs, o + I.r + I.nq + I.nc);
            o[I.d - 1] = c[row];
        }
        RET(upload(ctx, O + I.O_off, Op.data(), sizeof(double) * Op.size()));
        std::vector<double> PSt;
        if (I.rs) {
            std::vector<double> PS;
            PSt.resize((size_t)I.rs * I.nsdof);
            RET(to_host(ctx, PS, d.Phi_S, (size_t)I.nsdof * I.rs));
            for (int m = 0; m < I.nsdof; ++m)
                for (int k = 0; k < I.rs; ++k) PSt[(size_t)k * I.nsdof + m] = PS[(size_t)m * I.rs + k];
            RET(upload(ctx, PhiSt + I.PhiSt_off, PSt.data(), sizeof(double) * PSt.size()));
        }
        std::vector<short2> kk(std::max(1, I.nq));
        int t = 0;
        for (int a = 0; a < I.r; ++a)
            for (int b = a; b < I.r; ++b) kk[t++] = make_short2((short)a, (short)b);
        RET(upload(ctx, kij + I.kij_off, kk.data(), sizeof(short2) * I.nq));
        if (I.nc) {
            std::vector<short4> k3;
            k3.reserve(I.nc);
            for (int a = 0; a < I.r; ++a)
                for (int b = a; b < I.r; ++b)
                    for (int e = b; e < I.r; ++e) k3.push_back(make_short4((short)a, (short)b, (short)e, 0));
            RET(upload(ctx, kijk + I.kijk_off, k3.data(), sizeof(short4) * I.nc));
            CK(cudaStreamSynchronize(ctx->stream));  // k3 is a host staging buffer
        }
        // q0 = Phi^T u0, qd0 = Phi^T v0 over the free dofs
        RET(upload(ctx, uv, d.u0, sizeof(double) * 3 * nn));
        if (d.v0) RET(upload(ctx, uv + 3LL * nn, d.v0, sizeof(double) * 3 * nn));
        CK(launch_rom_basis_project(G.nfree[i], I.r, G.Phi[i], G.free_dof[i], uv, d.v0 ? uv + 3LL * nn : nullptr,
                                    B.q + I.q_off, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));  // host staging buffers and uv are reused
    }
    B.O = O;
    B.PhiSt = PhiSt;
    B.kij = kij;
    B.kijk = kijk;
    CKA(G.inst_d = ctx->alloc<InstRom>(n));
    RET(upload(ctx, G.inst_d, G.inst.data(), sizeof(InstRom) * n));
    B.inst = G.inst_d;
    CK(cudaStreamSynchronize(ctx->stream));
    return OSAM_OK;
}

int setup_couplings(osam_ctx* ctx, int n, const osam_problem_desc* descs,
                    const std::vector<std::vector<std::vector<uint8_t>>>& masks) {
    const int ncpl = descs[0].n_couplings;
    ctx->cpls.resize(ncpl);
    for (int k = 0; k < ncpl; ++k) {
        CplH& C = ctx->cpls[k];
        C.dst = descs[0].couplings[k].dst;
        C.src = descs[0].couplings[k].src;
        Slot& dst = ctx->slots[C.dst];
        Slot& src = ctx->slots[C.src];
        const bool dst_rom = dst.kind == OSAM_ROM, src_rom = src.kind == OSAM_ROM;
        std::vector<int> rinst, row, dnode_all, srcnode_local;
        std::vector<double> dw_all;
        std::vector<long long> rec_off(n), Rt_off(n), dst_hist_off(n);
        std::vector<int> dst_nd(n);
        C.nrow.assign(n, 0);
        C.row_first.assign(n, 0);
        long long rec_tot = 0, Rt_tot = 0;
        int* dn = nullptr;
        int* dnode_tmp = nullptr;
        double* dw_tmp = nullptr;
        size_t cap = 0;
        for (int i = 0; i < n; ++i) {
            const Grid& gd = dst_rom ? dst.rom.grid[i] : dst.fom.grid[i];
            const Grid& gs = src_rom ? src.rom.grid[i] : src.fom.grid[i];
            const std::vector<int>& srow_dst = dst_rom ? dst.rom.srow[i] : dst.fom.srow[i];
            std::vector<int> nodes;
            for (int nd = 0; nd < gd.nn(); ++nd)
                if (masks[i][k][nd]) nodes.push_back(nd);
            const int nr = (int)nodes.size();
            C.nrow[i] = nr;
            C.row_first[i] = (int)rinst.size();
            if (nodes.size() > cap) {
                cap = nodes.size();
                CKA(dn = ctx->alloc<int>(cap));
                CKA(dnode_tmp = ctx->alloc<int>(8 * cap));
                CKA(dw_tmp = ctx->alloc<double>(8 * cap));
            }
            std::vector<int> dnl(8 * nr);
            std::vector<double> dwl(8 * nr);
            if (nr) {
                RET(upload(ctx, dn, nodes.data(), sizeof(int) * nr));
                CK(cudaMemsetAsync(ctx->err_d, 0, sizeof(int), ctx->stream));
                CK(launch_donor(gs, gd, dn, nr, dnode_tmp, dw_tmp, ctx->err_d, ctx->stream));
                int nerr = 0;
                CK(cudaMemcpyAsync(&nerr, ctx->err_d, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
                CK(cudaMemcpyAsync(dnl.data(), dnode_tmp, sizeof(int) * 8 * nr, cudaMemcpyDeviceToHost, ctx->stream));
                CK(cudaMemcpyAsync(dwl.data(), dw_tmp, sizeof(double) * 8 * nr, cudaMemcpyDeviceToHost, ctx->stream));
                CK(cudaStreamSynchronize(ctx->stream));
                if (nerr)
                    return ctx->fail(OSAM_EDONOR, "instance %d coupling %d (%d <- %d): %d Schwarz nodes have no donor element",
                                     i, k, C.dst, C.src, nerr);
            }
            const long long src_off = src_rom ? 0 : src.fom.inst[i].node_off;
            for (int t = 0; t < nr; ++t) {
                rinst.push_back(i);
                row.push_back(srow_dst[nodes[t]]);
                for (int b = 0; b < 8; ++b) {
                    dnode_all.push_back((int)(src_off + dnl[8 * t + b]));
                    srcnode_local.push_back(dnl[8 * t + b]);
                    dw_all.push_back(dwl[8 * t + b]);
                }
            }
            rec_off[i] = rec_tot;
            rec_tot += (long long)(ctx->slots[C.src].nsub + 1) * 9 * nr;
            if (src_rom) {
                Rt_off[i] = Rt_tot;
                Rt_tot += (long long)src.rom.inst[i].r * 3 * nr;
            }
            dst_hist_off[i] = dst_rom ? dst.rom.inst[i].hist_off : dst.fom.inst[i].hist_off;
            dst_nd[i] = dst_rom ? dst.rom.inst[i].nsdof : dst.fom.inst[i].ns;
        }
        const int R = (int)rinst.size();
        CplB& B = C.d;
        B.R = R;
        B.dst_rom = dst_rom;
        B.dst_hist = dst_rom ? dst.rom.d.hist : dst.fom.d.hist;
        int* d_rinst = ctx->alloc<int>(R);
        int* d_row = ctx->alloc<int>(R);
        int* d_dnode = ctx->alloc<int>(8LL * R);
        double* d_dw = ctx->alloc<double>(8LL * R);
        int* d_first = ctx->alloc<int>(n);
        int* d_nrow = ctx->alloc<int>(n);
        long long* d_recoff = ctx->alloc<long long>(n);
        long long* d_rtoff = ctx->alloc<long long>(n);
        long long* d_dho = ctx->alloc<long long>(n);
        int* d_dnd = ctx->alloc<int>(n);
        CKA(d_rinst); CKA(d_row); CKA(d_dnode); CKA(d_dw); CKA(d_first); CKA(d_nrow); CKA(d_recoff); CKA(d_rtoff);
        CKA(d_dho); CKA(d_dnd);
        RET(upload(ctx, d_rinst, rinst.data(), sizeof(int) * R));
        RET(upload(ctx, d_row, row.data(), sizeof(int) * R));
        RET(upload(ctx, d_dnode, dnode_all.data(), sizeof(int) * 8 * R));
        RET(upload(ctx, d_dw, dw_all.data(), sizeof(double) * 8 * R));
        RET(upload(ctx, d_first, C.row_first.data(), sizeof(int) * n));
        RET(upload(ctx, d_nrow, C.nrow.data(), sizeof(int) * n));
        RET(upload(ctx, d_recoff, rec_off.data(), sizeof(long long) * n));
        RET(upload(ctx, d_rtoff, Rt_off.data(), sizeof(long long) * n));
        RET(upload(ctx, d_dho, dst_hist_off.data(), sizeof(long long) * n));
        RET(upload(ctx, d_dnd, dst_nd.data(), sizeof(int) * n));
        B.rinst = d_rinst; B.row = d_row; B.dnode = d_dnode; B.dw = d_dw; B.row_first = d_first; B.nrow = d_nrow;
        B.rec_off = d_recoff; B.Rt_off = d_rtoff; B.dst_hist_off = d_dho; B.dst_nd = d_dnd;
        if (!src_rom) {
            CKA(B.rec = ctx->alloc<double>(std::max(1LL, rec_tot)));
        } else {
            double* Rt = ctx->alloc<double>(std::max(1LL, Rt_tot));
            int* dloc = ctx->alloc<int>(8LL * std::max(1, R));
            CKA(Rt); CKA(dloc);
            RET(upload(ctx, dloc, srcnode_local.data(), sizeof(int) * 8 * R));
            CK(cudaMemsetAsync(ctx->err_d, 0, sizeof(int), ctx->stream));
            for (int i = 0; i < n; ++i) {
                const int f = C.row_first[i];
                CK(launch_build_Rt(C.nrow[i], src.rom.inst[i].r, dloc + 8LL * f, d_dw + 8LL * f, src.rom.dof_free[i],
                                   src.rom.srow_d[i], src.rom.Phi[i], Rt + Rt_off[i], ctx->err_d, ctx->stream));
            }
            int nerr = 0;
            CK(cudaMemcpyAsync(&nerr, ctx->err_d, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
            if (nerr)
                return ctx->fail(OSAM_EINVAL, "coupling %d: a donor node with nonzero weight is a Schwarz node of ROM %d", k,
                                 C.src);
            B.Rt = Rt;
        }
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return OSAM_OK;
}

int setup_controller(osam_ctx* ctx) {
    const int n = ctx->n_inst;
    CtlB& c = ctx->ctl;
    c.n_inst = n;
    c.ncpl = (int)ctx->cpls.size();
    c.max_it = ctx->max_it;
    c.tol_abs2 = ctx->tol_abs * ctx->tol_abs;
    c.tol_rel2 = ctx->tol_rel * ctx->tol_rel;
    c.n_fom = c.n_rom = 0;
    for (Slot& S : ctx->slots) {
        if (S.kind == OSAM_FOM) {
            c.fom_partial[c.n_fom] = S.fom.d.partial;
            c.fom_blk_off[c.n_fom] = S.fom.d.nblk_off;
            ++c.n_fom;
        } else {
            c.rom_npart[c.n_rom] = S.rom.d.npart;
            ++c.n_rom;
        }
    }
    CKA(c.active = ctx->alloc<int>(n));
    CKA(c.iters = ctx->alloc<int>(n));
    CKA(c.status = ctx->alloc<int>(n));
    CKA(c.cnum = ctx->alloc<double>(n));
    CKA(c.cden = ctx->alloc<double>(n));
    CKA(c.counter = ctx->alloc<unsigned int>(1));
    CKA(c.any_active = ctx->alloc<int>(1));
    CKA(ctx->sel = ctx->alloc<int>(n));
    CK(cudaMallocHost(&ctx->iters_h, sizeof(int) * n));
    CK(cudaMallocHost(&ctx->status_h, sizeof(int) * n));
    CK(cudaMallocHost(&ctx->cnum_h, sizeof(double) * n));
    CK(cudaMallocHost(&ctx->cden_h, sizeof(double) * n));
    CK(cudaMallocHost(&ctx->any_h, sizeof(int)));
    CK(cudaMallocHost(&ctx->imp_h, sizeof(int) * n));
    return OSAM_OK;
}

int select_instance(osam_ctx* ctx, int inst) {
    std::vector<int> sel(ctx->n_inst, 0);
    sel[inst] = 1;
    RET(upload(ctx, ctx->sel, sel.data(), sizeof(int) * ctx->n_inst));
    CK(cudaStreamSynchronize(ctx->stream));
    return OSAM_OK;
}

// initial accelerations of the instances selected by `mask` (null = all)
int initial_accel(osam_ctx* ctx, const int* mask) {
    for (Slot& S : ctx->slots) {
        if (S.kind == OSAM_FOM) {
            CK(launch_force_init_b(S.fom.d, mask, ctx->stream));
            CK(launch_init_accel_b(S.fom.d, mask, ctx->stream));
        } else {
            CK(launch_rom_project_b(S.rom.d, mask, 0, 0, ctx->stream));
            CK(launch_rom_step_b(S.rom.d, mask, 0, S.dt, 1, ctx->stream));
        }
    }
    return OSAM_OK;
}

// time force + node kernels of the largest FOM group for (element block, scatter) candidates on
// scratch copies of its state; keep the fastest (the deterministic gather scatter unless atomics are
// more than 5% faster)
int autotune(osam_ctx* ctx) {
    FomGroupH* best_g = nullptr;
    const Slot* best_s = nullptr;
    long long ne = -1;
    for (Slot& S : ctx->slots)
        if (S.kind == OSAM_FOM && S.fom.d.NE > ne) { ne = S.fom.d.NE; best_g = &S.fom; best_s = &S; }
    if (!best_g) return OSAM_OK;
    FomGroupH& G = *best_g;
    FomB g = G.d;
    const long long NN = g.NN;
    double *u = nullptr, *v = nullptr, *a = nullptr, *un = nullptr;
    CK(cudaMalloc(&u, sizeof(double) * 3 * NN));
    CK(cudaMalloc(&v, sizeof(double) * 3 * NN));
    CK(cudaMalloc(&a, sizeof(double) * 3 * NN));
    CK(cudaMalloc(&un, sizeof(double) * 3 * NN));
    CK(cudaMemcpyAsync(u, G.d.u[0], sizeof(double) * 3 * NN, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(v, G.d.v, sizeof(double) * 3 * NN, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(a, G.d.a, sizeof(double) * 3 * NN, cudaMemcpyDeviceToDevice, ctx->stream));
    g.v = v;
    g.a = a;
    const int slot2 = std::min(2, best_s->nsub);
    float best_ms = 1e30f, gather_ms = 1e30f;
    int best_block = 128, best_scatter = kGather, best_tiled = 0;
    // (scatter, element block, tiled).  The 128-register FP64 kernel measured level with the natural
    // one on the bench meshes, so AUTO does not try it (OSAM_SCATTER_GATHER_LOWREG selects it).
    const int cands[8][3] = {{kGather, 64, 0}, {kGather, 128, 0}, {kGather, 256, 0}, {kGather, 128, 1},
                             {kAtomic, 64, 0}, {kAtomic, 128, 0}, {kAtomic, 256, 0}, {kAtomic, 128, 1}};
    for (const auto& cd : cands) {
        const int mode = cd[0], block = cd[1], tiled = cd[2];
        if (g.df32 && (mode == kAtomic || block > 128 || tiled)) continue;  // double-float force: gather, <= 128 threads
        if (tiled && g.fp32) continue;                                    // the tiled kernel is FP64
        RET(set_eblocks(ctx, G, block));
        g.eblk = G.d.eblk;
        g.n_eblk = G.d.n_eblk;
        g.eblock = block;
        g.occ = 0;
        g.tiled = tiled;
        for (int rep = 0; rep < 4; ++rep) {
            if (rep == 1) CK(cudaEventRecord(ctx->ev0, ctx->stream));
            CK(launch_force_b(g, nullptr, mode, ctx->stream));
            CK(launch_node_b(g, nullptr, mode, 1, slot2, 0, u, un, best_s->dt, ctx->stream));
        }
        CK(cudaEventRecord(ctx->ev1, ctx->stream));
        CK(cudaEventSynchronize(ctx->ev1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
        if (mode == kGather) {
            if (ms < gather_ms) { gather_ms = ms; best_block = block; best_scatter = kGather; best_ms = ms; best_tiled = tiled; }
        } else if (ms < 0.95f * gather_ms && ms < best_ms) {
            best_ms = ms; best_block = block; best_scatter = kAtomic; best_tiled = tiled;
        }
    }
    CK(cudaMemsetAsync(G.d.f, 0, sizeof(double) * 3 * NN, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    cudaFree(u); cudaFree(v); cudaFree(a); cudaFree(un);
    ctx->scatter = best_scatter;
    for (Slot& S : ctx->slots)
        if (S.kind == OSAM_FOM) {
            RET(set_eblocks(ctx, S.fom, best_block));
            S.fom.d.tiled = best_tiled;
        }
    CK(cudaStreamSynchronize(ctx->stream));
    return OSAM_OK;
}

int init_impl(osam_ctx* ctx, int n, const osam_problem_desc* descs) {
    if (n < 1 || !descs) return ctx->fail(OSAM_EINVAL, "no instances");
    RET(validate_topology(ctx, n, descs));
    const osam_problem_desc& d0 = descs[0];
    RET(check_device(ctx, d0.device));
    ctx->device = d0.device;
    if (d0.stream) ctx->stream = static_cast<cudaStream_t>(d0.stream);
    else {
        int prio_lo = 0, prio_hi = 0;
        CK(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
        CK(cudaStreamCreateWithPriority(&ctx->stream, cudaStreamNonBlocking, prio_hi));
        ctx->own_stream = true;
    }
    ctx->n_inst = n;
    ctx->dt = d0.dt;
    ctx->nsub = d0.n_substeps;
    ctx->tol_abs = d0.tol_abs;
    ctx->tol_rel = d0.tol_rel;
    ctx->max_it = d0.max_iters;
    ctx->precision = d0.precision;
    ctx->scatter = (d0.scatter == OSAM_SCATTER_ATOMIC && d0.precision != OSAM_F32X2_FORCE) ? kAtomic : kGather;
    CK(cudaEventCreate(&ctx->ev0));
    CK(cudaEventCreate(&ctx->ev1));
    {
        int prio_lo = 0, prio_hi = 0;
        CK(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
        CK(cudaStreamCreateWithPriority(&ctx->side, cudaStreamNonBlocking, prio_lo));
        CK(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
        ctx->additive = d0.schwarz == OSAM_ADDITIVE;
        if (ctx->additive)
            for (int s = 1; s < d0.n_subdomains; ++s) {
                cudaStream_t l;
                cudaEvent_t e;
                CK(cudaStreamCreateWithPriority(&l, cudaStreamNonBlocking, prio_hi));
                ctx->lanes.push_back(l);
                CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
                ctx->lane_join.push_back(e);
            }
    }
    CKA(ctx->err_d = ctx->alloc<int>(1));
    const int nsd = d0.n_subdomains, ncpl = d0.n_couplings;
    ctx->slots.resize(nsd);
    ctx->fom_elements.assign(n, 0);
    // masks, Schwarz rows (union over the couplings into a subdomain, increasing node order)
    std::vector<std::vector<std::vector<uint8_t>>> masks(n, std::vector<std::vector<uint8_t>>(ncpl));
    int max_nn = 1;
    for (int s = 0; s < nsd; ++s) {
        Slot& S = ctx->slots[s];
        S.kind = d0.subdomains[s].kind;
        // Delta t_i = (dt n_substeps) / n_i; exactly dt for the common count
        const int ni = d0.subdomains[s].n_substeps;
        S.nsub = ni > 0 ? ni : ctx->nsub;
        S.dt = S.nsub == ctx->nsub ? ctx->dt : (ctx->dt * (double)ctx->nsub) / (double)S.nsub;
    }
    for (int i = 0; i < n; ++i) {
        const osam_problem_desc& d = descs[i];
        for (int s = 0; s < nsd; ++s) {
            const osam_subdomain_desc& sd = d.subdomains[s];
            Grid g;
            g.nx = sd.nx; g.ny = sd.ny; g.nz = sd.nz; g.h = sd.h;
            for (int a = 0; a < 3; ++a) g.org[a] = sd.origin[a];
            const int nn = g.nn();
            max_nn = std::max(max_nn, nn);
            std::vector<uint8_t> clamp(nn, 0);
            if (sd.dirichlet) CK(cudaMemcpy(clamp.data(), sd.dirichlet, nn, cudaMemcpyDefault));
            for (auto& c : clamp) c &= 7;
            Slot& S = ctx->slots[s];
            if (S.kind == OSAM_FOM) {
                S.fom.grid.push_back(g);
                S.fom.clamp.push_back(clamp);
                ctx->fom_elements[i] += (long long)g.ne() * S.nsub;
            } else {
                S.rom.grid.push_back(g);
                S.rom.clamp.push_back(clamp);
            }
        }
        for (int k = 0; k < ncpl; ++k) {
            const osam_coupling_desc& c = d.couplings[k];
            const Slot& S = ctx->slots[c.dst];
            const int nn = (S.kind == OSAM_FOM ? S.fom.grid[i] : S.rom.grid[i]).nn();
            masks[i][k].resize(nn);
            CK(cudaMemcpy(masks[i][k].data(), c.nodes, nn, cudaMemcpyDefault));
        }
        for (int s = 0; s < nsd; ++s) {
            Slot& S = ctx->slots[s];
            const int nn = (S.kind == OSAM_FOM ? S.fom.grid[i] : S.rom.grid[i]).nn();
            std::vector<int> srow(nn, -1);
            int ns = 0;
            for (int nd = 0; nd < nn; ++nd) {
                bool any = false;
                for (int k = 0; k < ncpl; ++k)
                    if (d.couplings[k].dst == s && masks[i][k][nd]) any = true;
                if (any) srow[nd] = ns++;
            }
            if (S.kind == OSAM_FOM) { S.fom.srow.push_back(srow); S.fom.ns.push_back(ns); }
            else { S.rom.srow.push_back(srow); S.rom.ns.push_back(ns); }
        }
    }
    CKA(ctx->scratch = ctx->alloc<double>(3LL * max_nn));
    for (int s = 0; s < nsd; ++s) {
        Slot& S = ctx->slots[s];
        if (S.kind == OSAM_FOM) RET(setup_fom_group(ctx, S.fom, s, n, descs));
        else RET(setup_rom_group(ctx, S.rom, s, n, descs));
    }
    RET(setup_couplings(ctx, n, descs, masks));
    if (ctx->any_implicit)
        for (cudaStream_t& c : ctx->cap) CK(cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking));
    RET(setup_controller(ctx));
    // initial boundary data: zero-order hold of the initial states (before the accelerations)
    for (CplH& c : ctx->cpls) RET(zoh_cpl(ctx, c, nullptr));
    RET(initial_accel(ctx, nullptr));
    if (d0.scatter == OSAM_SCATTER_AUTO) RET(autotune(ctx));
    if (d0.scatter == OSAM_SCATTER_GATHER_LOWREG && d0.precision == OSAM_FP64)
        for (Slot& S : ctx->slots)
            if (S.kind == OSAM_FOM) S.fom.d.occ = 1;
    if (d0.scatter == OSAM_SCATTER_GATHER_TILED && d0.precision == OSAM_FP64)
        for (Slot& S : ctx->slots)
            if (S.kind == OSAM_FOM) S.fom.d.tiled = 1;
    for (Slot& S : ctx->slots)
        if (S.kind == OSAM_FOM) S.fom.d.scatter = ctx->scatter;
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->launches = 0;
    return OSAM_OK;
}

bool valid(osam_ctx* ctx, int inst, int sub) {
    return ctx && inst >= 0 && inst < ctx->n_inst && sub >= 0 && sub < (int)ctx->slots.size();
}

}  // namespace

extern "C" {

const char* osam_last_error(const osam_ctx* ctx) {
    if (!ctx) return g_init_error.c_str();
    return ctx->err.c_str();
}

int osam_scatter_mode(osam_ctx* ctx) { return ctx ? ctx->scatter : 0; }

int osam_tuning(osam_ctx* ctx, int* scatter, int* element_block, int* register_cap, int* tiled) {
    if (!ctx) return OSAM_EINVAL;
    if (scatter) *scatter = ctx->scatter;
    if (tiled) {
        *tiled = 0;
        for (Slot& S : ctx->slots)
            if (S.kind == OSAM_FOM && S.fom.d.tiled) *tiled = 1;
    }
    if (register_cap) {
        *register_cap = 0;
        for (Slot& S : ctx->slots)
            if (S.kind == OSAM_FOM && S.fom.d.occ) *register_cap = 128;
    }
    if (element_block) {
        *element_block = 0;
        for (Slot& S : ctx->slots)
            if (S.kind == OSAM_FOM) *element_block = S.fom.d.eblock;
    }
    return OSAM_OK;
}

int osam_num_instances(osam_ctx* ctx) { return ctx ? ctx->n_inst : 0; }

int osam_set_graph(osam_ctx* ctx, int enable) {
    if (!ctx) return OSAM_EINVAL;
    ctx->use_graph = enable != 0;
    return OSAM_OK;
}

void osam_destroy(osam_ctx* ctx) { delete ctx; }

int osam_batch_init(int n_instances, const osam_problem_desc* descs, osam_ctx** out) {
    if (out) *out = nullptr;
    g_init_error.clear();
    if (!descs || !out || n_instances < 1) { g_init_error = "null argument"; return OSAM_EINVAL; }
    auto* ctx = new osam_ctx();
    int rc = init_impl(ctx, n_instances, descs);
    if (rc != OSAM_OK) {
        g_init_error = ctx->err;
        delete ctx;
        return rc;
    }
    *out = ctx;
    return OSAM_OK;
}

int schwarz_init(const osam_problem_desc* desc, osam_ctx** out) { return osam_batch_init(1, desc, out); }

int subdomain_advance(osam_ctx* ctx, int sub) {
    if (!valid(ctx, 0, sub)) return OSAM_EINVAL;
    RET(advance_slot(ctx, sub, nullptr));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->prof_collect();
    return OSAM_OK;
}

int transfer_overlap(osam_ctx* ctx, int src, int dst) {
    if (!ctx) return OSAM_EINVAL;
    bool any = false;
    for (CplH& c : ctx->cpls)
        if (c.src == src && c.dst == dst) {
            any = true;
            RET(transfer_cpl(ctx, c, nullptr));
        }
    if (!any) return ctx->fail(OSAM_EINVAL, "no coupling %d -> %d", src, dst);
    CK(cudaStreamSynchronize(ctx->stream));
    return OSAM_OK;
}

int osam_begin_interval(osam_ctx* ctx) {
    if (!ctx) return OSAM_EINVAL;
    RET(enqueue_begin(ctx));
    CK(cudaStreamSynchronize(ctx->stream));
    return OSAM_OK;
}

int osam_restore_interval(osam_ctx* ctx) {
    if (!ctx) return OSAM_EINVAL;
    RET(saverest_all(ctx, nullptr, 1));
    CK(cudaStreamSynchronize(ctx->stream));
    return OSAM_OK;
}

int osam_criterion(osam_ctx* ctx, double* cnum, double* cden) {
    if (!ctx) return OSAM_EINVAL;
    LK(launch_reset_ctl(ctx->ctl, ctx->stream));
    RET(norms_all(ctx, nullptr));
    LK(launch_controller(ctx->ctl, ctx->cond, 0, ctx->stream));
    RET(read_ctl(ctx));
    CK(cudaStreamSynchronize(ctx->stream));
    if (cnum) *cnum = ctx->cnum_h[0];
    if (cden) *cden = ctx->cden_h[0];
    if (ctx->status_h[0] == OSAM_ENONFINITE) return ctx->fail(OSAM_ENONFINITE, "non-finite coupled state");
    return OSAM_OK;
}

int osam_batch_step(osam_ctx* ctx, osam_step_report* reps, osam_step_report* total) {
    if (!ctx) return OSAM_EINVAL;
    const bool graph = ctx->use_graph && !ctx->prof;
    if (graph) RET(build_graph(ctx));
    CK(cudaEventRecord(ctx->ev0, ctx->stream));
    if (graph) {
        CK(cudaGraphLaunch(ctx->exec, ctx->stream));
    } else {
        RET(enqueue_begin(ctx));
        for (int n = 1; n <= ctx->max_it; ++n) {
            RET(enqueue_iteration(ctx, 0));
            CK(cudaMemcpyAsync(ctx->any_h, ctx->ctl.any_active, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
            if (!*ctx->any_h) break;
        }
    }
    CK(cudaEventRecord(ctx->ev1, ctx->stream));
    RET(read_ctl(ctx));
    CK(cudaEventSynchronize(ctx->ev1));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->prof_collect();
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
    int worst = OSAM_OK, max_its = 0;
    long long updates = 0;
    for (int i = 0; i < ctx->n_inst; ++i) {
        const int st = ctx->status_h[i];
        if (st < 0) worst = std::min(worst, st);
        else if (worst >= 0) worst = std::max(worst, st);
        max_its = std::max(max_its, ctx->iters_h[i]);
        const long long u = (long long)ctx->iters_h[i] * ctx->fom_elements[i];
        updates += u;
        if (reps) {
            reps[i].status = st;
            reps[i].iterations = ctx->iters_h[i];
            reps[i].cnum = ctx->cnum_h[i];
            reps[i].cden = ctx->cden_h[i];
            reps[i].element_updates = u;
            reps[i].elapsed_ms = ms;
        }
    }
    if (graph) ctx->launches += ctx->graph_begin_launches + (long long)max_its * ctx->graph_body_launches;
    if (total) {
        total->status = worst;
        total->iterations = max_its;
        total->cnum = ctx->cnum_h[0];
        total->cden = ctx->cden_h[0];
        total->element_updates = updates;
        total->elapsed_ms = ms;
    }
    if (worst == OSAM_ENONFINITE) return ctx->fail(OSAM_ENONFINITE, "non-finite coupled state");
    return worst;
}

int schwarz_step(osam_ctx* ctx, osam_step_report* rep) {
    if (!ctx) return OSAM_EINVAL;
    if (ctx->n_inst == 1) return osam_batch_step(ctx, rep, nullptr);
    return osam_batch_step(ctx, nullptr, rep);
}

int osam_profile(osam_ctx* ctx, int enable) {
    if (!ctx) return OSAM_EINVAL;
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->prof_collect();
    ctx->prof = enable != 0;
    ctx->prof_ms = ctx->tprof_ms = 0.0;
    ctx->prof_launches = ctx->prof_elements = ctx->tprof_launches = 0;
    ctx->launches = 0;
    for (Slot& S : ctx->slots)
        if (S.kind == OSAM_FOM && S.fom.d.implicit)
            CK(cudaMemsetAsync(S.fom.d.istat, 0, sizeof(long long) * 2 * S.fom.d.n_inst, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return OSAM_OK;
}

int osam_implicit_profile(osam_ctx* ctx, double* tangent_ms, long long* tangent_launches,
                          long long* tangent_elements, long long* newton_steps, long long* cg_iterations) {
    if (!ctx) return OSAM_EINVAL;
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->prof_collect();
    long long el = 0, nw = 0, cg = 0;
    for (Slot& S : ctx->slots) {
        if (S.kind != OSAM_FOM || !S.fom.d.implicit) continue;
        std::vector<long long> st;
        RET(to_host(ctx, st, S.fom.d.istat, 2 * (size_t)S.fom.d.n_inst));
        for (int i = 0; i < S.fom.d.n_inst; ++i) {
            nw += st[2 * i];
            cg += st[2 * i + 1];
            el += st[2 * i + 1] * S.fom.inst[i].ne;
        }
    }
    if (tangent_ms) *tangent_ms = ctx->tprof_ms;
    if (tangent_launches) *tangent_launches = ctx->tprof_launches;
    if (tangent_elements) *tangent_elements = el;
    if (newton_steps) *newton_steps = nw;
    if (cg_iterations) *cg_iterations = cg;
    return OSAM_OK;
}

int osam_profile_read(osam_ctx* ctx, double* force_ms, long long* force_launches, long long* force_elements,
                      long long* kernel_launches) {
    if (!ctx) return OSAM_EINVAL;
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->prof_collect();
    if (force_ms) *force_ms = ctx->prof_ms;
    if (force_launches) *force_launches = ctx->prof_launches;
    if (force_elements) *force_elements = ctx->prof_elements;
    if (kernel_launches) *kernel_launches = ctx->launches;
    return OSAM_OK;
}

int osam_instance_sizes(osam_ctx* ctx, int inst, int sub, int* n_nodes, int* n_elements, int* n_free,
                        int* n_schwarz) {
    if (!valid(ctx, inst, sub)) return OSAM_EINVAL;
    Slot& S = ctx->slots[sub];
    const Grid& g = S.kind == OSAM_FOM ? S.fom.grid[inst] : S.rom.grid[inst];
    const std::vector<uint8_t>& cl = S.kind == OSAM_FOM ? S.fom.clamp[inst] : S.rom.clamp[inst];
    const std::vector<int>& sr = S.kind == OSAM_FOM ? S.fom.srow[inst] : S.rom.srow[inst];
    if (n_nodes) *n_nodes = g.nn();
    if (n_elements) *n_elements = g.ne();
    if (n_schwarz) *n_schwarz = S.kind == OSAM_FOM ? S.fom.ns[inst] : S.rom.ns[inst];
    if (n_free) {
        int nf = 0;
        for (int nd = 0; nd < g.nn(); ++nd)
            for (int c = 0; c < 3; ++c) nf += !(cl[nd] & (1 << c)) && sr[nd] < 0;
        *n_free = nf;
    }
    return OSAM_OK;
}

int osam_sizes(osam_ctx* ctx, int sub, int* n_nodes, int* n_elements, int* n_free, int* n_schwarz) {
    return osam_instance_sizes(ctx, 0, sub, n_nodes, n_elements, n_free, n_schwarz);
}

int osam_instance_get_state(osam_ctx* ctx, int inst, int sub, double* u, double* v, double* a) {
    if (!valid(ctx, inst, sub)) return OSAM_EINVAL;
    Slot& S = ctx->slots[sub];
    double* outs[3] = {u, v, a};
    for (int f = 0; f < 3; ++f) {
        if (!outs[f]) continue;
        int nn;
        if (S.kind == OSAM_FOM) {
            const InstFom& I = S.fom.inst[inst];
            nn = I.nn;
            const double* src = f == 0 ? S.fom.d.u[0] : (f == 1 ? S.fom.d.v : S.fom.d.a);
            CK(launch_soa_to_aos(src + I.node_off, ctx->scratch, nn, S.fom.d.NN, ctx->stream));
        } else {
            RomGroupH& G = S.rom;
            const InstRom& I = G.inst[inst];
            nn = G.grid[inst].nn();
            const double* hs = G.d.hist + I.hist_off + ((long long)S.nsub * 3 + f) * I.nsdof;
            CK(launch_rom_full_field(nn, I.r, G.Phi[inst], G.dof_free[inst], G.clamp_d[inst], G.srow_d[inst], hs,
                                     G.d.q + I.q_off + (long long)f * I.r, ctx->scratch, ctx->stream));
        }
        CK(cudaMemcpyAsync(outs[f], ctx->scratch, sizeof(double) * 3 * nn, cudaMemcpyDefault, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return OSAM_OK;
}

int osam_get_state(osam_ctx* ctx, int sub, double* u, double* v, double* a) {
    return osam_instance_get_state(ctx, 0, sub, u, v, a);
}

int osam_instance_set_state(osam_ctx* ctx, int inst, int sub, const double* u, const double* v, const double* a) {
    if (!valid(ctx, inst, sub) || !u) return OSAM_EINVAL;
    Slot& S = ctx->slots[sub];
    if (S.kind == OSAM_FOM) {
        FomB& g = S.fom.d;
        const InstFom& I = S.fom.inst[inst];
        RET(upload(ctx, ctx->scratch, u, sizeof(double) * 3 * I.nn));
        CK(launch_aos_to_soa(ctx->scratch, g.u[0] + I.node_off, I.nn, g.NN, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        if (v) {
            RET(upload(ctx, ctx->scratch, v, sizeof(double) * 3 * I.nn));
            CK(launch_aos_to_soa(ctx->scratch, g.v + I.node_off, I.nn, g.NN, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
        } else {
            for (int c = 0; c < 3; ++c)
                CK(cudaMemsetAsync(g.v + c * g.NN + I.node_off, 0, sizeof(double) * I.nn, ctx->stream));
        }
        CK(launch_zero_clamped(I.nn, g.clamp + I.node_off, g.u[0] + I.node_off, g.v + I.node_off, g.NN, ctx->stream));
        if (a) {
            RET(upload(ctx, ctx->scratch, a, sizeof(double) * 3 * I.nn));
            CK(launch_aos_to_soa(ctx->scratch, g.a + I.node_off, I.nn, g.NN, ctx->stream));
        } else {
            RET(select_instance(ctx, inst));
            CK(launch_force_init_b(g, ctx->sel, ctx->stream));
            CK(launch_init_accel_b(g, ctx->sel, ctx->stream));
        }
    } else {
        RomGroupH& G = S.rom;
        const InstRom& I = G.inst[inst];
        const int nn = G.grid[inst].nn();
        std::vector<double> qh(I.r), qdh(I.r, 0.0);
        RET(upload(ctx, ctx->scratch, u, sizeof(double) * 3 * nn));
        CK(launch_rom_basis_project(G.nfree[inst], I.r, G.Phi[inst], G.free_dof[inst], ctx->scratch, nullptr,
                                    G.d.q + I.q_off, ctx->stream));
        RET(to_host(ctx, qh, G.d.q + I.q_off, I.r));
        if (v) {
            RET(upload(ctx, ctx->scratch, v, sizeof(double) * 3 * nn));
            CK(launch_rom_basis_project(G.nfree[inst], I.r, G.Phi[inst], G.free_dof[inst], ctx->scratch, nullptr,
                                        G.d.q + I.q_off, ctx->stream));
            RET(to_host(ctx, qdh, G.d.q + I.q_off, I.r));
        }
        RET(upload(ctx, G.d.q + I.q_off, qh.data(), sizeof(double) * I.r));
        RET(upload(ctx, G.d.q + I.q_off + I.r, qdh.data(), sizeof(double) * I.r));
        RET(select_instance(ctx, inst));
        CK(launch_rom_project_b(G.d, ctx->sel, 0, 0, ctx->stream));
        CK(launch_rom_step_b(G.d, ctx->sel, 0, S.dt, 1, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return OSAM_OK;
}

int osam_set_state(osam_ctx* ctx, int sub, const double* u, const double* v, const double* a) {
    return osam_instance_set_state(ctx, 0, sub, u, v, a);
}

int osam_instance_get_reduced_state(osam_ctx* ctx, int inst, int sub, double* q, double* qd, double* qdd) {
    if (!valid(ctx, inst, sub) || ctx->slots[sub].kind != OSAM_ROM) return OSAM_EINVAL;
    RomGroupH& G = ctx->slots[sub].rom;
    const InstRom& I = G.inst[inst];
    double* outs[3] = {q, qd, qdd};
    for (int f = 0; f < 3; ++f)
        if (outs[f])
            CK(cudaMemcpyAsync(outs[f], G.d.q + I.q_off + (long long)f * I.r, sizeof(double) * I.r, cudaMemcpyDefault,
                               ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return OSAM_OK;
}

int osam_get_reduced_state(osam_ctx* ctx, int sub, double* q, double* qd, double* qdd) {
    return osam_instance_get_reduced_state(ctx, 0, sub, q, qd, qdd);
}

int osam_instance_set_reduced_state(osam_ctx* ctx, int inst, int sub, const double* q, const double* qd,
                                    const double* qdd) {
    if (!valid(ctx, inst, sub) || ctx->slots[sub].kind != OSAM_ROM) return OSAM_EINVAL;
    RomGroupH& G = ctx->slots[sub].rom;
    const InstRom& I = G.inst[inst];
    const double* ins[3] = {q, qd, qdd};
    for (int f = 0; f < 3; ++f)
        if (ins[f])
            CK(cudaMemcpyAsync(G.d.q + I.q_off + (long long)f * I.r, ins[f], sizeof(double) * I.r, cudaMemcpyDefault,
                               ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return OSAM_OK;
}

int osam_set_reduced_state(osam_ctx* ctx, int sub, const double* q, const double* qd, const double* qdd) {
    return osam_instance_set_reduced_state(ctx, 0, sub, q, qd, qdd);
}

// ------------------------------------------------------------------------------------------------
// element-level operators
// ------------------------------------------------------------------------------------------------
static ElemArgs standalone_args(int nx, int ny, int nz, double h, double lambda, double mu, const double* lam_e,
                                const double* mu_e, const double* u) {
    ElemArgs a{};
    a.nx = nx; a.ny = ny; a.nz = nz; a.ne = nx * ny * nz;
    a.invh = 1.0 / h;
    a.w8 = h * h / 8.0;
    a.lam = lambda; a.mu = mu;
    a.lam_e = lam_e; a.mu_e = mu_e;
    a.u = u; a.usn = 3; a.usc = 1;
    a.fsn = 3; a.fsc = 1;
    return a;
}

int osam_hex8_force(int nx, int ny, int nz, double h, int material, double lambda, double mu, const double* lambda_e,
                    const double* mu_e, const double* u, double* f, void* stream) {
    if (nx < 1 || ny < 1 || nz < 1 || !(h > 0.0) || !u || !f) return OSAM_EINVAL;
    if (material != OSAM_LINEAR_ELASTIC && material != OSAM_NEO_HOOKEAN && material != OSAM_SAINT_VENANT_KIRCHHOFF)
        return OSAM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long nn = (long long)(nx + 1) * (ny + 1) * (nz + 1);
    if (cudaMemsetAsync(f, 0, sizeof(double) * 3 * nn, s) != cudaSuccess) return OSAM_ECUDA;
    ElemArgs a = standalone_args(nx, ny, nz, h, lambda, mu, lambda_e, mu_e, u);
    a.f = f;
    return launch_hex8_force(material, false, kAtomic, a, s) == cudaSuccess ? OSAM_OK : OSAM_ECUDA;
}

int osam_hex8_force_vjp(int nx, int ny, int nz, double h, int material, double lambda, double mu,
                        const double* lambda_e, const double* mu_e, const double* u, const double* ybar, double* ubar,
                        double* lambda_bar, double* mu_bar, void* stream) {
    if (nx < 1 || ny < 1 || nz < 1 || !(h > 0.0) || !u || !ybar || !ubar) return OSAM_EINVAL;
    if (material != OSAM_LINEAR_ELASTIC && material != OSAM_NEO_HOOKEAN) return OSAM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long nn = (long long)(nx + 1) * (ny + 1) * (nz + 1);
    if (cudaMemsetAsync(ubar, 0, sizeof(double) * 3 * nn, s) != cudaSuccess) return OSAM_ECUDA;
    ElemArgs a = standalone_args(nx, ny, nz, h, lambda, mu, lambda_e, mu_e, u);
    a.f = ubar;
    return launch_hex8_vjp(material, a, ybar, 3, 1, lambda_bar, mu_bar, 0, s) == cudaSuccess ? OSAM_OK : OSAM_ECUDA;
}

// ------------------------------------------------------------------------------------------------
// adjoint rollout on a one-instance FOM group without couplings
// ------------------------------------------------------------------------------------------------
int osam_adjoint(const osam_adjoint_desc* d, osam_adjoint_out* out) {
    if (!d || !out) return OSAM_EINVAL;
    if (d->nx < 1 || d->ny < 1 || d->nz < 1 || !(d->h > 0.0) || !d->u0 || !d->w || !d->lambda_e || !d->mu_e ||
        d->n_steps < 0 || !(d->dt > 0.0) || !(d->rho > 0.0) ||
        (d->material != OSAM_LINEAR_ELASTIC && d->material != OSAM_NEO_HOOKEAN))
        return OSAM_EINVAL;
    osam_subdomain_desc sd{};
    sd.kind = OSAM_FOM;
    sd.nx = d->nx; sd.ny = d->ny; sd.nz = d->nz; sd.h = d->h;
    sd.material = d->material;
    sd.rho = d->rho;
    sd.lambda_e = d->lambda_e; sd.mu_e = d->mu_e;
    sd.dirichlet = d->dirichlet;
    sd.u0 = d->u0; sd.v0 = d->v0;
    osam_problem_desc pd{};
    pd.n_subdomains = 1;
    pd.subdomains = &sd;
    pd.dt = d->dt;
    pd.n_substeps = 1;
    pd.max_iters = 1;
    pd.precision = OSAM_FP64;
    pd.scatter = OSAM_SCATTER_ATOMIC;
    pd.stream = d->stream;
    pd.device = d->device;
    osam_ctx* raw = nullptr;
    if (int rc = osam_batch_init(1, &pd, &raw)) return rc;
    std::unique_ptr<osam_ctx> holder(raw);
    osam_ctx* ctx = raw;
    FomB& F = ctx->slots[0].fom.d;
    const InstFom& I = ctx->slots[0].fom.inst[0];
    const int nn = I.nn, ne = I.ne;
    const double dt = d->dt;
    const int T = d->n_steps;
    const int Cp = d->checkpoint_every > 0 ? d->checkpoint_every : 50;
    const int nck = T / Cp + 1;
    const long long n3 = 3LL * nn;
    double* ck = ctx->alloc<double>((size_t)nck * 3 * n3);  // (u, v, a) at steps 0, C, 2C, ...
    double* useg = ctx->alloc<double>((size_t)(Cp + 1) * n3);
    double* ub = ctx->alloc<double>(n3);
    double* vb = ctx->alloc<double>(n3);
    double* ab = ctx->alloc<double>(n3);
    double* y = ctx->alloc<double>(n3);
    double* tmp = ctx->alloc<double>(n3);
    double* glam = ctx->alloc<double>(ne);
    double* gmu = ctx->alloc<double>(ne);
    CKA(ck); CKA(useg); CKA(ub); CKA(vb); CKA(ab); CKA(y); CKA(tmp); CKA(glam); CKA(gmu);
    CK(cudaEventRecord(ctx->ev0, ctx->stream));
    // one explicit step in place on (u[0], v, a)
    auto step = [&](double* u_store) -> int {
        CK(launch_node_b(F, nullptr, kAtomic, -1, 1, 1, F.u[0], F.u[1], dt, ctx->stream));
        CK(launch_force_b(F, nullptr, kAtomic, ctx->stream));
        CK(launch_node_b(F, nullptr, kAtomic, 1, -1, 0, F.u[1], F.u[0], dt, ctx->stream));
        CK(cudaMemcpyAsync(F.u[0], F.u[1], sizeof(double) * n3, cudaMemcpyDeviceToDevice, ctx->stream));
        if (u_store) CK(cudaMemcpyAsync(u_store, F.u[0], sizeof(double) * n3, cudaMemcpyDeviceToDevice, ctx->stream));
        return OSAM_OK;
    };
    auto save_ck = [&](int idx) -> int {
        double* base = ck + (size_t)idx * 3 * n3;
        CK(cudaMemcpyAsync(base, F.u[0], sizeof(double) * n3, cudaMemcpyDeviceToDevice, ctx->stream));
        CK(cudaMemcpyAsync(base + n3, F.v, sizeof(double) * n3, cudaMemcpyDeviceToDevice, ctx->stream));
        CK(cudaMemcpyAsync(base + 2 * n3, F.a, sizeof(double) * n3, cudaMemcpyDeviceToDevice, ctx->stream));
        return OSAM_OK;
    };
    auto load_ck = [&](int idx) -> int {
        double* base = ck + (size_t)idx * 3 * n3;
        CK(cudaMemcpyAsync(F.u[0], base, sizeof(double) * n3, cudaMemcpyDeviceToDevice, ctx->stream));
        CK(cudaMemcpyAsync(F.v, base + n3, sizeof(double) * n3, cudaMemcpyDeviceToDevice, ctx->stream));
        CK(cudaMemcpyAsync(F.a, base + 2 * n3, sizeof(double) * n3, cudaMemcpyDeviceToDevice, ctx->stream));
        return OSAM_OK;
    };
    RET(save_ck(0));
    for (int t = 1; t <= T; ++t) {
        RET(step(nullptr));
        if (t % Cp == 0) RET(save_ck(t / Cp));
    }
    // J = w . u_T
    RET(upload(ctx, ctx->scratch, d->w, sizeof(double) * n3));
    CK(launch_aos_to_soa(ctx->scratch, ub, nn, nn, ctx->stream));
    CK(launch_zero_clamped(nn, F.clamp, ub, nullptr, nn, ctx->stream));
    std::vector<double> wh(n3), uh(n3);
    CK(cudaMemcpyAsync(wh.data(), ub, sizeof(double) * n3, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(uh.data(), F.u[0], sizeof(double) * n3, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    double J = 0.0;
    for (long long q = 0; q < n3; ++q) J += wh[q] * uh[q];
    ElemArgs va{};
    va.nx = I.nx; va.ny = I.ny; va.nz = I.nz; va.ne = ne;
    va.invh = I.invh; va.w8 = I.w8;
    va.lam_e = I.lam_e; va.mu_e = I.mu_e;
    va.usn = 1; va.usc = nn; va.fsn = 1; va.fsc = nn;
    va.f = tmp;
    for (int seg = (T - 1) / Cp; seg >= 0 && T > 0; --seg) {
        const int t0 = seg * Cp, t1 = std::min(T, t0 + Cp);
        RET(load_ck(seg));
        CK(cudaMemcpyAsync(useg, F.u[0], sizeof(double) * n3, cudaMemcpyDeviceToDevice, ctx->stream));
        for (int t = t0 + 1; t <= t1; ++t) RET(step(useg + (size_t)(t - t0) * n3));
        for (int t = t1 - 1; t >= t0; --t) {
            CK(launch_adjoint_pre(nn, dt, F.clamp, F.minv, vb, ab, y, tmp, ctx->stream));
            va.u = useg + (size_t)(t + 1 - t0) * n3;
            CK(launch_hex8_vjp(F.material, va, y, 1, nn, glam, gmu, 1, ctx->stream));
            CK(launch_adjoint_post(nn, dt, F.clamp, tmp, ub, vb, ab, ctx->stream));
        }
    }
    // a_0 = -M^-1 f(u_0)
    CK(launch_adjoint_pre(nn, 0.0, F.clamp, F.minv, vb, ab, y, tmp, ctx->stream));
    RET(load_ck(0));
    va.u = F.u[0];
    CK(launch_hex8_vjp(F.material, va, y, 1, nn, glam, gmu, 1, ctx->stream));
    CK(launch_adjoint_post(nn, 0.0, F.clamp, tmp, ub, vb, ab, ctx->stream));
    CK(cudaEventRecord(ctx->ev1, ctx->stream));
    CK(cudaEventSynchronize(ctx->ev1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
    out->J = J;
    out->elapsed_ms = ms;
    if (out->grad_u0) {
        CK(launch_soa_to_aos(ub, ctx->scratch, nn, nn, ctx->stream));
        CK(cudaMemcpyAsync(out->grad_u0, ctx->scratch, sizeof(double) * n3, cudaMemcpyDefault, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    if (out->grad_v0) {
        CK(launch_soa_to_aos(vb, ctx->scratch, nn, nn, ctx->stream));
        CK(cudaMemcpyAsync(out->grad_v0, ctx->scratch, sizeof(double) * n3, cudaMemcpyDefault, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    if (out->grad_lambda) CK(cudaMemcpyAsync(out->grad_lambda, glam, sizeof(double) * ne, cudaMemcpyDefault, ctx->stream));
    if (out->grad_mu) CK(cudaMemcpyAsync(out->grad_mu, gmu, sizeof(double) * ne, cudaMemcpyDefault, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return OSAM_OK;
}

}  // extern "C"
