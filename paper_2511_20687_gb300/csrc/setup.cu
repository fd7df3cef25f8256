// Set-up of libosam's host runtime: validation of the problem descriptions, the device data of every
// FOM and ROM group (meshes, lumped masses, node sets, material tables, tiles, ROM operators and their
// Kronecker index tables), the couplings (donor search, trilinear weights, trace and history buffers),
// the controller state, the initial accelerations and the launch autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ctx.h"

namespace osam {
namespace host {

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
    if (d0.precision != OSAM_FP64 && d0.precision != OSAM_FP32_FORCE && d0.precision != OSAM_F32X2_FORCE &&
        d0.precision != OSAM_FP64_TANGENT32)
        return ctx->fail(OSAM_EINVAL, "bad precision");
    if (d0.scatter < OSAM_SCATTER_AUTO || d0.scatter > OSAM_SCATTER_GATHER_TILED_LOWREG)
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
            if (a.kind == OSAM_FOM && a.integrator == OSAM_IMPLICIT && d0.precision != OSAM_FP64 &&
                d0.precision != OSAM_FP64_TANGENT32)
                return ctx->fail(OSAM_EINVAL,
                                 "subdomain %d: implicit integration needs OSAM_FP64 or OSAM_FP64_TANGENT32", s);
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
        I.wq = g.h * g.h / 32.0;
        I.wq3 = g.h * g.h / 96.0;
        I.lam = d.lambda; I.mu = d.mu;
        if (d.material == OSAM_NEO_HOOKEAN) {
            const double kappa = d.lambda + (2.0 / 3.0) * d.mu;
            I.m1 = 0.5 * kappa * I.wq; I.m2 = d.mu * I.wq; I.m3 = d.mu * I.wq3;
        } else {
            I.m1 = d.lambda * I.wq; I.m2 = d.mu * I.wq; I.m3 = 0.0;
        }
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
    if (B.df32 || B.fp32) CKA(B.u2 = ctx->alloc<float2>(3 * NN));   // the FP32 forces' split of u/h
    B.implicit = descs[0].subdomains[s].integrator == OSAM_IMPLICIT;
    if (B.implicit) {
        ctx->any_implicit = true;
        CKA(B.ut = ctx->alloc<double>(3 * NN));
        CKA(B.cg_x = ctx->alloc<double>(3 * NN));
        CKA(B.cg_r = ctx->alloc<double>(3 * NN));
        CKA(B.cg_p = ctx->alloc<double>(3 * NN));
        CKA(B.cg_ap = ctx->alloc<double>(3 * NN));
        double* mass = ctx->alloc<double>(NN);
        CKA(mass);
        B.mass = mass;
        for (double** p : {&B.rn2, &B.r0, &B.rr, &B.rrn, &B.rr0, &B.pap, &B.cgtol2, &B.alpha, &B.beta})
            CKA(*p = ctx->alloc<double>(n));
        CKA(B.iticket = ctx->alloc<unsigned int>(n));
        CK(cudaMemsetAsync(B.iticket, 0, sizeof(unsigned int) * n, ctx->stream));
        CKA(B.istat = ctx->alloc<long long>(2 * n));
        CKA(B.iloop = ctx->alloc<int>(2));
        if (B.material == OSAM_NEO_HOOKEAN && ctx->precision == OSAM_FP64_TANGENT32) {
            CKA(B.linf = ctx->alloc<float>((long long)kLinPerGp * 8 * NE));
            CKA(B.fe32 = ctx->alloc<float>(24 * NE));
        } else if (B.material == OSAM_NEO_HOOKEAN) {
            CKA(B.lin = ctx->alloc<double>((long long)kLinPerGp * 8 * NE));
        }
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
        CK(launch_lumped_minv(G.grid[i], d.rho, minv + I.node_off, ctx->stream,
                              B.mass ? const_cast<double*>(B.mass) + I.node_off : nullptr));
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
    if (B.df32 || B.fp32) CK(launch_split_u2_b(B, ctx->stream));
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
    struct Scratch {   // the candidates' state copies, freed on every return path
        double* p[4] = {nullptr, nullptr, nullptr, nullptr};
        ~Scratch() { for (double* q : p) cudaFree(q); }
    } sc;
    for (double*& q : sc.p) CK(cudaMalloc(&q, sizeof(double) * 3 * NN));
    double *u = sc.p[0], *v = sc.p[1], *a = sc.p[2], *un = sc.p[3];
    CK(cudaMemcpyAsync(u, G.d.u[0], sizeof(double) * 3 * NN, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(v, G.d.v, sizeof(double) * 3 * NN, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(a, G.d.a, sizeof(double) * 3 * NN, cudaMemcpyDeviceToDevice, ctx->stream));
    g.v = v;
    g.a = a;
    const int slot2 = std::min(2, best_s->nsub);
    float best_ms = 1e30f, gather_ms = 1e30f;
    int best_block = 128, best_scatter = kGather, best_tiled = 0, best_occ = 0;
    // (scatter, element block, tiled, 128-register cap).  Both FP64 kernels capped at 128 registers
    // measured level with their natural builds on the bench meshes (tiled: 192.8 vs 193.1 us per launch
    // on 40x40x80, the fourth resident tile per SM paid for by its spills), so AUTO does not try them
    // (OSAM_SCATTER_GATHER_LOWREG / _TILED_LOWREG select them).
    const int cands[8][4] = {{kGather, 64, 0, 0}, {kGather, 128, 0, 0}, {kGather, 256, 0, 0}, {kGather, 128, 1, 0},
                             {kAtomic, 64, 0, 0}, {kAtomic, 128, 0, 0}, {kAtomic, 256, 0, 0}, {kAtomic, 128, 1, 0}};
    for (const auto& cd : cands) {
        const int mode = cd[0], block = cd[1], tiled = cd[2], occ = cd[3];
        if (g.df32 && (mode == kAtomic || block > 128 || tiled)) continue;  // double-float force: gather, <= 128 threads
        if (tiled && g.fp32) continue;                                    // the tiled kernel is FP64
        RET(set_eblocks(ctx, G, block));
        g.eblk = G.d.eblk;
        g.n_eblk = G.d.n_eblk;
        g.eblock = block;
        g.occ = occ;
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
            if (ms < gather_ms) {
                gather_ms = ms; best_block = block; best_scatter = kGather; best_ms = ms; best_tiled = tiled; best_occ = occ;
            }
        } else if (ms < 0.95f * gather_ms && ms < best_ms) {
            best_ms = ms; best_block = block; best_scatter = kAtomic; best_tiled = tiled; best_occ = 0;
        }
    }
    CK(cudaMemsetAsync(G.d.f, 0, sizeof(double) * 3 * NN, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->scatter = best_scatter;
    for (Slot& S : ctx->slots)
        if (S.kind == OSAM_FOM) {
            RET(set_eblocks(ctx, S.fom, best_block));
            S.fom.d.tiled = best_tiled;
            S.fom.d.occ = best_occ;
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
    const bool fp64_force = d0.precision == OSAM_FP64 || d0.precision == OSAM_FP64_TANGENT32;
    if (d0.scatter == OSAM_SCATTER_GATHER_LOWREG && fp64_force)
        for (Slot& S : ctx->slots)
            if (S.kind == OSAM_FOM) S.fom.d.occ = 1;
    if ((d0.scatter == OSAM_SCATTER_GATHER_TILED || d0.scatter == OSAM_SCATTER_GATHER_TILED_LOWREG) && fp64_force)
        for (Slot& S : ctx->slots)
            if (S.kind == OSAM_FOM) {
                S.fom.d.tiled = 1;
                S.fom.d.occ = d0.scatter == OSAM_SCATTER_GATHER_TILED_LOWREG;
            }
    for (Slot& S : ctx->slots)
        if (S.kind == OSAM_FOM) S.fom.d.scatter = ctx->scatter;
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->launches = 0;
    return OSAM_OK;
}

}  // namespace host
}  // namespace osam
