// O-SAM controller of libosam's host runtime: the per-step kernel sequences of Algorithm 1 (FOM
// substeps with fused overlap traces, ROM substeps, transfers through the temporal interpolant,
// criterion of Eq. conv_criterion), the multiplicative and additive sweeps, the implicit intervals
// (Newton / CG as device-side loops) and the controller step as one CUDA graph.  Only sequences and
// checks: every numerical step runs in the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ctx.h"

namespace osam {
namespace host {

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
constexpr double kCgTol2F32 = 1e-12;   // the floor with the FP32 tangent (eta >= 1e-6, above its rounding)

// the stored-linearisation path (Neo-Hookean groups), and the CG floor that goes with its precision
bool stored_lin(const FomB& g) { return g.lin || g.linf; }
double cg_floor(const FomB& g) { return g.linf ? kCgTol2F32 : kCgTol2; }

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
            if (stored_lin(g)) LK(launch_force_lin_b(g, g.nact, ctx->stream));
            else LK(launch_force_b(g, g.nact, kGather, ctx->stream, nullptr));
            LK(launch_imp_residual_b(g, g.nact, c0, ctx->stream));
            LK(launch_imp_reduce_b(g, g.nact, 0, it == 0, kNewtonTol2, ctx->stream));
            bool any = false;
            RET(any_set(ctx, g.nact, n, any));
            if (!any) break;
            for (int k = 0; k < kCgMax;) {
                for (int q = 0; q < kCgCheck; ++q, ++k) {
                    const int pk = ctx->prof_begin(1);
                    if (stored_lin(g)) LK(launch_tangent_lin_b(g, g.cgact, ctx->stream));
                    else LK(launch_tangent_b(g, g.cgact, ctx->stream));
                    ctx->prof_end(pk, 0);
                    LK(launch_cg_ap_b(g, g.cgact, c0, ctx->stream));
                    LK(launch_cg_step_b(g, g.cgact, c0, cg_floor(g), ctx->stream));
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
                if (stored_lin(g)) LK(launch_force_lin_b(g, g.nact, a));
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
                    if (stored_lin(g)) LK(launch_tangent_lin_b(g, g.cgact, b));
                    else LK(launch_tangent_b(g, g.cgact, b));
                    LK(launch_cg_ap_b(g, g.cgact, c0, b));
                    LK(launch_cg_step_b(g, g.cgact, c0, cg_floor(g), b));
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

}  // namespace host
}  // namespace osam
