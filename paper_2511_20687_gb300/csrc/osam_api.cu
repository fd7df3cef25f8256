// C ABI of libosam (include/osam.h): context construction for one problem or a batch of instances
// (schwarz_init / osam_batch_init), the controller entry points, state I/O, measurement hooks, the
// element-level operators and the adjoint rollout.  The runtime itself is in setup.cu and
// controller.cu; this file checks arguments, calls it and reports errors.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <functional>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "ctx.h"

namespace {
thread_local std::string g_init_error;
}  // namespace

namespace osam {
void set_thread_error(const std::string& msg) { g_init_error = msg; }
}  // namespace osam

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
        // a device-accessible buffer (this device's memory, mapped page-locked host memory) is written
        // in place by the layout kernel; anything else through the staging buffer and a copy
        double* direct = static_cast<double*>(direct_view(ctx, outs[f]));
        double* dst = direct ? direct : ctx->scratch;
        int nn;
        if (S.kind == OSAM_FOM) {
            const InstFom& I = S.fom.inst[inst];
            nn = I.nn;
            const double* src = f == 0 ? S.fom.d.u[0] : (f == 1 ? S.fom.d.v : S.fom.d.a);
            CK(launch_soa_to_aos(src + I.node_off, dst, nn, S.fom.d.NN, ctx->stream));
        } else {
            RomGroupH& G = S.rom;
            const InstRom& I = G.inst[inst];
            nn = G.grid[inst].nn();
            const double* hs = G.d.hist + I.hist_off + ((long long)S.nsub * 3 + f) * I.nsdof;
            CK(launch_rom_full_field(nn, I.r, G.Phi[inst], G.dof_free[inst], G.clamp_d[inst], G.srow_d[inst], hs,
                                     G.d.q + I.q_off + (long long)f * I.r, dst, ctx->stream));
        }
        // stream order lets the next field reuse the staging buffer; one host synchronisation at the end
        if (!direct)
            CK(cudaMemcpyAsync(outs[f], ctx->scratch, sizeof(double) * 3 * nn, cudaMemcpyDefault, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return OSAM_OK;
}

int osam_get_state(osam_ctx* ctx, int sub, double* u, double* v, double* a) {
    return osam_instance_get_state(ctx, 0, sub, u, v, a);
}

int osam_instance_set_state(osam_ctx* ctx, int inst, int sub, const double* u, const double* v, const double* a) {
    if (!valid(ctx, inst, sub) || !u) return OSAM_EINVAL;
    Slot& S = ctx->slots[sub];
    const double* src = nullptr;
    if (S.kind == OSAM_FOM) {
        FomB& g = S.fom.d;
        const InstFom& I = S.fom.inst[inst];
        // the staging buffer is reused in stream order; the caller's buffers are released by the final
        // synchronisation
        RET(stage_in(ctx, u, 3 * (size_t)I.nn, &src));
        CK(launch_aos_to_soa(src, g.u[0] + I.node_off, I.nn, g.NN, ctx->stream));
        if (v) {
            RET(stage_in(ctx, v, 3 * (size_t)I.nn, &src));
            CK(launch_aos_to_soa(src, g.v + I.node_off, I.nn, g.NN, ctx->stream));
        } else {
            for (int c = 0; c < 3; ++c)
                CK(cudaMemsetAsync(g.v + c * g.NN + I.node_off, 0, sizeof(double) * I.nn, ctx->stream));
        }
        CK(launch_zero_clamped(I.nn, g.clamp + I.node_off, g.u[0] + I.node_off, g.v + I.node_off, g.NN, ctx->stream));
        if (a) {
            RET(stage_in(ctx, a, 3 * (size_t)I.nn, &src));
            CK(launch_aos_to_soa(src, g.a + I.node_off, I.nn, g.NN, ctx->stream));
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
        RET(stage_in(ctx, u, 3 * (size_t)nn, &src));
        CK(launch_rom_basis_project(G.nfree[inst], I.r, G.Phi[inst], G.free_dof[inst], src, nullptr,
                                    G.d.q + I.q_off, ctx->stream));
        RET(to_host(ctx, qh, G.d.q + I.q_off, I.r));
        if (v) {
            RET(stage_in(ctx, v, 3 * (size_t)nn, &src));
            CK(launch_rom_basis_project(G.nfree[inst], I.r, G.Phi[inst], G.free_dof[inst], src, nullptr,
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
    a.wq = h * h / 32.0;
    a.wq3 = h * h / 96.0;
    a.lam = lambda; a.mu = mu;
    a.lam_e = lam_e; a.mu_e = mu_e;
    a.u = u; a.usn = 3; a.usc = 1;
    a.fsn = 3; a.fsc = 1;
    return a;
}

// mesh sizes the element-level kernels index with 32-bit element and node numbers
static bool elem_mesh_ok(const char* who, int nx, int ny, int nz, double h) {
    if (nx < 1 || ny < 1 || nz < 1 || !(h > 0.0)) {
        set_thread_error(std::string(who) + ": mesh dimensions and h must be positive");
        return false;
    }
    const long long ne = (long long)nx * ny * nz;   // < 2^93 cannot wrap in the node product below
    const double nn = (double(nx) + 1.0) * (double(ny) + 1.0) * (double(nz) + 1.0);
    if (ne > INT_MAX || 3.0 * nn > double(INT_MAX)) {
        set_thread_error(std::string(who) + ": mesh too large for 32-bit element / node indices");
        return false;
    }
    return true;
}

int osam_hex8_force(int nx, int ny, int nz, double h, int material, double lambda, double mu, const double* lambda_e,
                    const double* mu_e, const double* u, double* f, void* stream) {
    if (!elem_mesh_ok("osam_hex8_force", nx, ny, nz, h)) return OSAM_EINVAL;
    if (!u || !f) {
        set_thread_error("osam_hex8_force: u and f must be device pointers");
        return OSAM_EINVAL;
    }
    if (material != OSAM_LINEAR_ELASTIC && material != OSAM_NEO_HOOKEAN && material != OSAM_SAINT_VENANT_KIRCHHOFF) {
        set_thread_error("osam_hex8_force: unknown material");
        return OSAM_EINVAL;
    }
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
    if (!elem_mesh_ok("osam_hex8_force_vjp", nx, ny, nz, h)) return OSAM_EINVAL;
    if (!u || !ybar || !ubar) {
        set_thread_error("osam_hex8_force_vjp: u, ybar and ubar must be device pointers");
        return OSAM_EINVAL;
    }
    if (material != OSAM_LINEAR_ELASTIC && material != OSAM_NEO_HOOKEAN) {
        set_thread_error("osam_hex8_force_vjp: material must be linear elastic or Neo-Hookean");
        return OSAM_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long nn = (long long)(nx + 1) * (ny + 1) * (nz + 1);
    if (cudaMemsetAsync(ubar, 0, sizeof(double) * 3 * nn, s) != cudaSuccess) return OSAM_ECUDA;
    ElemArgs a = standalone_args(nx, ny, nz, h, lambda, mu, lambda_e, mu_e, u);
    a.f = ubar;
    return launch_hex8_vjp(material, kAtomic, a, ybar, 3, 1, lambda_bar, mu_bar, 0, s) == cudaSuccess ? OSAM_OK
                                                                                              : OSAM_ECUDA;
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
    pd.scatter = OSAM_SCATTER_GATHER;   // element buffer + fixed-order gather: bitwise repeatable gradients
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
    double* useg[2] = {ctx->alloc<double>((size_t)(Cp + 1) * n3), ctx->alloc<double>((size_t)(Cp + 1) * n3)};
    double* ub = ctx->alloc<double>(n3);
    double* vb = ctx->alloc<double>(n3);
    double* ab = ctx->alloc<double>(n3);
    double* y = ctx->alloc<double>(n3);
    double* vfe = ctx->alloc<double>(24LL * ne);   // the VJP's element buffer (the recomputation uses F.fe)
    double* glam = ctx->alloc<double>(ne);
    double* gmu = ctx->alloc<double>(ne);
    CKA(ck); CKA(useg[0]); CKA(useg[1]); CKA(ub); CKA(vb); CKA(ab); CKA(y); CKA(vfe); CKA(glam); CKA(gmu);
    const cudaStream_t R = ctx->stream;   // forward sweep and reverse sweeps (the critical path)
    const cudaStream_t Q = ctx->side;     // recomputation of the next segment, concurrently
    struct Events {
        cudaEvent_t e[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
        ~Events() { for (auto x : e) if (x) cudaEventDestroy(x); }
    } ev;
    for (auto& x : ev.e) CK(cudaEventCreateWithFlags(&x, cudaEventDisableTiming));
    cudaEvent_t ev_rec[2] = {ev.e[0], ev.e[1]}, ev_rev[2] = {ev.e[2], ev.e[3]}, ev_start = ev.e[4];
    CK(cudaEventRecord(ctx->ev0, R));
    // one explicit step in place on (u[0], v, a), deterministic element-buffer scatter
    auto step = [&](double* u_store, cudaStream_t st) -> int {
        CK(launch_node_b(F, nullptr, kGather, -1, 1, 1, F.u[0], F.u[1], dt, st));
        CK(launch_force_b(F, nullptr, kGather, st));
        CK(launch_node_b(F, nullptr, kGather, 1, -1, 0, F.u[1], F.u[0], dt, st));
        CK(cudaMemcpyAsync(F.u[0], F.u[1], sizeof(double) * n3, cudaMemcpyDeviceToDevice, st));
        if (u_store) CK(cudaMemcpyAsync(u_store, F.u[0], sizeof(double) * n3, cudaMemcpyDeviceToDevice, st));
        return OSAM_OK;
    };
    auto save_ck = [&](int idx) -> int {
        double* base = ck + (size_t)idx * 3 * n3;
        CK(cudaMemcpyAsync(base, F.u[0], sizeof(double) * n3, cudaMemcpyDeviceToDevice, R));
        CK(cudaMemcpyAsync(base + n3, F.v, sizeof(double) * n3, cudaMemcpyDeviceToDevice, R));
        CK(cudaMemcpyAsync(base + 2 * n3, F.a, sizeof(double) * n3, cudaMemcpyDeviceToDevice, R));
        return OSAM_OK;
    };
    auto load_ck = [&](int idx, cudaStream_t st) -> int {
        double* base = ck + (size_t)idx * 3 * n3;
        CK(cudaMemcpyAsync(F.u[0], base, sizeof(double) * n3, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(F.v, base + n3, sizeof(double) * n3, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(F.a, base + 2 * n3, sizeof(double) * n3, cudaMemcpyDeviceToDevice, st));
        return OSAM_OK;
    };
    ElemArgs va{};
    va.nx = I.nx; va.ny = I.ny; va.nz = I.nz; va.ne = ne;
    va.invh = I.invh; va.w8 = I.w8; va.wq = I.wq; va.wq3 = I.wq3;
    va.lam_e = I.lam_e; va.mu_e = I.mu_e;
    va.usn = 1; va.usc = nn;
    va.fe = vfe;
    // reverse of step t + 1 of a segment starting at t0 (state u_{t+1} stored at buf[t + 1 - t0])
    auto reverse = [&](int t, int t0, const double* buf, cudaStream_t st) -> int {
        CK(launch_adjoint_pre(nn, dt, F.clamp, F.minv, vb, ab, y, st));
        va.u = buf + (size_t)(t + 1 - t0) * n3;
        CK(launch_hex8_vjp(F.material, kGather, va, y, 1, nn, glam, gmu, 1, st));
        CK(launch_adjoint_post(I.nx, I.ny, I.nz, dt, F.clamp, vfe, ub, vb, ab, st));
        return OSAM_OK;
    };
    // A full segment of Cp steps is the same sequence of launches every time (the checkpoint is loaded
    // outside it and the segment buffers are reused), so the forward sweep, the recomputation into
    // either buffer and the reverse sweep from either buffer are each captured once as a CUDA graph and
    // replayed; a partial last segment runs from the host.
    struct Graphs {
        cudaGraphExec_t g[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
        ~Graphs() { for (auto x : g) if (x) cudaGraphExecDestroy(x); }
    } graphs;
    auto capture = [&](int which, const std::function<int()>& body) -> int {
        cudaGraph_t gr = nullptr;
        CK(cudaStreamBeginCapture(R, cudaStreamCaptureModeThreadLocal));
        const int rc = body();
        const cudaError_t e = cudaStreamEndCapture(R, &gr);
        if (rc) { if (gr) cudaGraphDestroy(gr); return rc; }
        CK(e);
        const cudaError_t ei = cudaGraphInstantiate(&graphs.g[which], gr, 0);
        cudaGraphDestroy(gr);
        CK(ei);
        return OSAM_OK;
    };
    if (T >= Cp) {
        RET(capture(0, [&]() -> int { for (int t = 0; t < Cp; ++t) RET(step(nullptr, R)); return OSAM_OK; }));
        for (int b = 0; b < 2; ++b) {
            RET(capture(1 + b, [&]() -> int {
                CK(cudaMemcpyAsync(useg[b], F.u[0], sizeof(double) * n3, cudaMemcpyDeviceToDevice, R));
                for (int t = 1; t <= Cp; ++t) RET(step(useg[b] + (size_t)t * n3, R));
                return OSAM_OK;
            }));
            RET(capture(3 + b, [&]() -> int {
                for (int t = Cp - 1; t >= 0; --t) RET(reverse(t, 0, useg[b], R));
                return OSAM_OK;
            }));
        }
    }
    RET(save_ck(0));
    for (int t0 = 0; t0 < T; t0 += Cp) {
        if (t0 + Cp <= T) {
            CK(cudaGraphLaunch(graphs.g[0], R));
            RET(save_ck((t0 + Cp) / Cp));
        } else {
            for (int t = t0 + 1; t <= T; ++t) RET(step(nullptr, R));
        }
    }
    // J = w . u_T
    RET(upload(ctx, ctx->scratch, d->w, sizeof(double) * n3));
    CK(launch_aos_to_soa(ctx->scratch, ub, nn, nn, R));
    CK(launch_zero_clamped(nn, F.clamp, ub, nullptr, nn, R));
    std::vector<double> wh(n3), uh(n3);
    CK(cudaMemcpyAsync(wh.data(), ub, sizeof(double) * n3, cudaMemcpyDeviceToHost, R));
    CK(cudaMemcpyAsync(uh.data(), F.u[0], sizeof(double) * n3, cudaMemcpyDeviceToHost, R));
    CK(cudaStreamSynchronize(R));
    double J = 0.0;
    for (long long q = 0; q < n3; ++q) J += wh[q] * uh[q];
    // Reverse sweep.  A partial last segment is recomputed and reversed on R first.  Then the full
    // segments s = S-1 .. 0: the recomputation of segment s - 1 needs only checkpoint s - 1, so it runs
    // on Q into the other buffer while the reverse sweep of segment s runs on R.  Buffer s % 2 is
    // rewritten only after the reverse sweep that last read it (segment s + 2) is done.
    int seg = T > 0 ? (T - 1) / Cp : -1;
    if (seg >= 0 && T - seg * Cp < Cp) {
        const int t0 = seg * Cp;
        RET(load_ck(seg, R));
        CK(cudaMemcpyAsync(useg[0], F.u[0], sizeof(double) * n3, cudaMemcpyDeviceToDevice, R));
        for (int t = t0 + 1; t <= T; ++t) RET(step(useg[0] + (size_t)(t - t0) * n3, R));
        for (int t = T - 1; t >= t0; --t) RET(reverse(t, t0, useg[0], R));
        --seg;
    }
    if (seg >= 0) {
        CK(cudaEventRecord(ev_start, R));
        CK(cudaStreamWaitEvent(Q, ev_start, 0));
        RET(load_ck(seg, Q));
        CK(cudaGraphLaunch(graphs.g[1 + seg % 2], Q));
        CK(cudaEventRecord(ev_rec[seg % 2], Q));
        for (int sg = seg; sg >= 0; --sg) {
            CK(cudaStreamWaitEvent(R, ev_rec[sg % 2], 0));
            CK(cudaGraphLaunch(graphs.g[3 + sg % 2], R));
            CK(cudaEventRecord(ev_rev[sg % 2], R));
            if (sg > 0) {
                if (sg + 1 <= seg) CK(cudaStreamWaitEvent(Q, ev_rev[(sg - 1) % 2], 0));   // segment sg + 1's
                RET(load_ck(sg - 1, Q));
                CK(cudaGraphLaunch(graphs.g[1 + (sg - 1) % 2], Q));
                CK(cudaEventRecord(ev_rec[(sg - 1) % 2], Q));
            }
        }
    }
    // a_0 = -M^-1 f(u_0) (Q has no work left: every recomputation finished before its reverse sweep)
    CK(launch_adjoint_pre(nn, 0.0, F.clamp, F.minv, vb, ab, y, R));
    RET(load_ck(0, R));
    va.u = F.u[0];
    CK(launch_hex8_vjp(F.material, kGather, va, y, 1, nn, glam, gmu, 1, R));
    CK(launch_adjoint_post(I.nx, I.ny, I.nz, 0.0, F.clamp, vfe, ub, vb, ab, R));
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
