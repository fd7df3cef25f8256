// Implicit Newmark subdomains (average acceleration, beta = 1/4, gamma = 1/2, the implicit member of
// the Newmark family of Sec. 4.1), batched over the instances of a FOM group like the explicit
// kernels.  Per substep:
//   predictor  u~ = u + dt v + (1/2 - beta) dt^2 a on free dofs, Dirichlet / Schwarz data elsewhere;
//   Newton     R(u) = M (u - u~) / (beta dt^2) + f_int(u) = 0 on the free dofs; each Newton system
//              J du = -R, J = M / (beta dt^2) + K(u), solved by conjugate gradients preconditioned
//              with the mass term, J applied matrix-free: K(u) p is the directional derivative of the
//              element forces (Appendix A tangents) in the force kernels' sum factorisation;
//   corrector  a = (u - u~) / (beta dt^2), v += dt ((1 - gamma) a_old + gamma a).
// Every inner product is reduced per node block, then per instance in a fixed order (deterministic).
// Newton and CG activity is tracked per instance on the device; the host reads it to stop.
#include <cuda_runtime.h>

#include <cstdint>

#include "hex8_math.cuh"
#include "osam_internal.h"

namespace osam {

namespace {

using namespace hex8;

__device__ __forceinline__ bool run(const int* mask, int inst) { return !mask || mask[inst]; }

__device__ __forceinline__ double block_sum1(double x) {
    __shared__ double sx[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    const int w = threadIdx.x / 32, l = threadIdx.x % 32;
    __syncthreads();
    if (l == 0) sx[w] = x;
    __syncthreads();
    double a = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)((blockDim.x + 31) / 32); ++i) a += sx[i];
    return a;
}

struct NodeCtx {
    int inst, n;
    long long gn;
    InstFom I;
    bool ok;
};

__device__ __forceinline__ NodeCtx node_ctx(const FomB& g, const int* mask) {
    NodeCtx c;
    const int2 b = g.nblk[blockIdx.x];
    c.inst = b.x;
    c.I = g.inst[b.x];
    c.n = b.y + threadIdx.x;
    c.gn = c.I.node_off + c.n;
    c.ok = run(mask, b.x) && c.n < c.I.nn;
    return c;
}

__device__ __forceinline__ bool is_free(const FomB& g, long long gn, int c) {
    return !(g.clamp[gn] & (1 << c)) && g.srow[gn] < 0;
}

// predictor and boundary data of the new level; u lives in u[0] for implicit groups
__global__ void __launch_bounds__(kNodeBlock) k_imp_predict_b(const FomB g, const int* __restrict__ active, int slot1,
                                                              double dt) {
    const NodeCtx x = node_ctx(g, active);
    if (!x.ok) return;
    const uint8_t cm = g.clamp[x.gn];
    const int row = g.srow[x.gn];
    const double* h1 = g.hist + x.I.hist_off + (long long)slot1 * 9 * x.I.ns;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const long long d = (long long)c * g.NN + x.gn;
        double u;
        if (cm & (1 << c)) u = 0.0;
        else if (row >= 0) u = h1[(long long)c * x.I.ns + row];
        else u = g.u[0][d] + dt * g.v[d] + (0.25 * dt * dt) * g.a[d];
        g.u[0][d] = u;
        g.ut[d] = u;
        g.us[d] = u * x.I.invh;
    }
}

// R = M (u - ut) c0 + f (free dofs; the element forces of u are in the element buffer).  CG start
// x = 0, r = -R, z = p = M^-1 r / c0 (the mass part of the tangent as preconditioner); partials
// |R|^2 and r . z
__global__ void __launch_bounds__(kNodeBlock) k_imp_residual_b(const FomB g, const int* __restrict__ mask, double c0,
                                                               double ic0) {
    const NodeCtx x = node_ctx(g, mask);
    double s = 0.0, sz = 0.0;
    if (x.ok) {
        const int i = x.n % (x.I.nx + 1);
        const int t = x.n / (x.I.nx + 1);
        const int j = t % (x.I.ny + 1);
        const int k = t / (x.I.ny + 1);
        const double* fe = static_cast<const double*>(g.fe) + x.I.elem_off;
        const double m = g.mass[x.gn];
        const double pz = g.minv[x.gn] * ic0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long d = (long long)c * g.NN + x.gn;
            double R = 0.0;
            if (is_free(g, x.gn, c)) {
                const double f = gather_force<double>(fe, x.I.nx, x.I.ny, x.I.nz, (int)g.NE, i, j, k, c);
                R = c0 * m * (g.u[0][d] - g.ut[d]) + f;
            }
            g.cg_x[d] = 0.0;
            g.cg_r[d] = -R;
            g.cg_p[d] = -R * pz;
            s = fma(R, R, s);
            sz = fma(R * pz, R, sz);
        }
    }
    s = block_sum1(s);
    sz = block_sum1(sz);
    if (threadIdx.x == 0) {
        g.ipart[blockIdx.x] = s;
        g.ipart[g.n_nblk + blockIdx.x] = sz;
    }
}

// per-instance fixed-order sums of the node-block partials, and the decisions that depend on them
__global__ void k_imp_reduce_b(const FomB g, const int* __restrict__ mask, int mode, int first, double tol2) {
    const int inst = blockIdx.x;
    if (!run(mask, inst)) return;
    if (first < 0) first = g.iloop[0] == 0;  // device-side Newton loop: its counter says which step this is
    const int b0 = g.nblk_off[inst], b1 = g.nblk_off[inst + 1];
    double s = 0.0, sz = 0.0;
    for (int b = b0 + (int)threadIdx.x; b < b1; b += blockDim.x) {
        s += g.ipart[b];
        sz += g.ipart[g.n_nblk + b];
    }
    s = block_sum1(s);
    sz = block_sum1(sz);
    if (threadIdx.x != 0) return;
    if (mode == 0) {
        if (first) g.r0[inst] = s;
        // forcing term of the inexact Newton step (Eisenstat and Walker's second choice, gamma = 1,
        // alpha = 2): relative CG tolerance eta = min(1e-6, (|R_k| / |R_k-1|)^2), never below the CG
        // floor of k_cg_step_b; stored squared, as r . z is compared squared-norm to squared-norm
        double eta2 = 1e-12;
        if (!first && g.rn2[inst] > 0.0) {
            const double ratio2 = s / g.rn2[inst];
            eta2 = fmin(1e-12, ratio2 * ratio2);
        }
        g.cgtol2[inst] = eta2;
        g.rn2[inst] = s;
        g.rr[inst] = sz;
        g.rr0[inst] = sz;
        const bool fin = isfinite(s) && isfinite(sz);
        const int st = !fin ? 2 : ((s == 0.0 || s <= tol2 * g.r0[inst]) ? 0 : 1);
        g.nact[inst] = st;
        g.cgact[inst] = st == 1 ? 1 : 0;
        if (st == 1) g.istat[2 * inst] += 1;
    } else {
        // mode 3: |du|^2 against |u|^2 after the update: an increment at the rounding level of u converges
        if (isfinite(s) && s <= tol2 * sz) g.nact[inst] = 0;
    }
}

// The last node block of an instance to finish sums the instance's block partials, in the fixed
// order of k_imp_reduce_b (same arithmetic, so the fused kernels reproduce the separate reductions
// bit for bit).  Called by every thread of the block; true in thread 0 of the last block, with the sum.
__device__ __forceinline__ bool last_block_sum(const FomB& g, int inst, double& total) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int t = atomicAdd(g.iticket + inst, 1u);
        last = t == (unsigned int)(g.nblk_off[inst + 1] - g.nblk_off[inst] - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    const int b0 = g.nblk_off[inst], b1 = g.nblk_off[inst + 1];
    double s = 0.0;
    for (int b = b0 + (int)threadIdx.x; b < b1; b += blockDim.x) s += __ldcg(g.ipart + b);
    s = block_sum1(s);
    if (threadIdx.x != 0) return false;
    g.iticket[inst] = 0u;
    total = s;
    return true;
}

// K p at node (i, j, k), component c, from the FP32 element buffer of the FP32 tangent: the 8 corner
// contributions summed in FP32 in the fixed order of gather_force, converted once
__device__ __forceinline__ double gather_tangent32(const float* fe, int nx, int ny, int nz, int ne, int i, int j,
                                                   int k, int c) {
    float s = 0.f;
#pragma unroll
    for (int az = 0; az < 2; ++az) {
        const int ke = k - az;
        if (ke < 0 || ke >= nz) continue;
#pragma unroll
        for (int ay = 0; ay < 2; ++ay) {
            const int je = j - ay;
            if (je < 0 || je >= ny) continue;
#pragma unroll
            for (int ax = 0; ax < 2; ++ax) {
                const int ie = i - ax;
                if (ie < 0 || ie >= nx) continue;
                s += __ldg(fe + (long long)((ax + 2 * ay + 4 * az) * 3 + c) * ne + (ie + nx * (je + ny * ke)));
            }
        }
    }
    return double(s);
}

// Ap = M p c0 + K p (free dofs; K p from the FP64 element buffer, or the FP32 one of the FP32 tangent);
// p . Ap summed per instance by its last block, which sets alpha = (r . z) / (p . Ap) for the step kernel
__global__ void __launch_bounds__(kNodeBlock) k_cg_ap_b(const FomB g, const int* __restrict__ mask, double c0) {
    const NodeCtx x = node_ctx(g, mask);
    double s = 0.0;
    if (x.ok) {
        const int i = x.n % (x.I.nx + 1);
        const int t = x.n / (x.I.nx + 1);
        const int j = t % (x.I.ny + 1);
        const int k = t / (x.I.ny + 1);
        const double* fe = static_cast<const double*>(g.fe) + x.I.elem_off;
        const float* fe32 = g.fe32 ? g.fe32 + x.I.elem_off : nullptr;
        const double m = g.mass[x.gn];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long d = (long long)c * g.NN + x.gn;
            double ap = 0.0;
            if (is_free(g, x.gn, c)) {
                const double kp = fe32 ? gather_tangent32(fe32, x.I.nx, x.I.ny, x.I.nz, (int)g.NE, i, j, k, c)
                                       : gather_force<double>(fe, x.I.nx, x.I.ny, x.I.nz, (int)g.NE, i, j, k, c);
                ap = c0 * m * g.cg_p[d] + kp;
            }
            g.cg_ap[d] = ap;
            s = fma(g.cg_p[d], ap, s);
        }
    }
    s = block_sum1(s);
    if (threadIdx.x == 0) g.ipart[blockIdx.x] = s;
    double pap;
    if (last_block_sum(g, x.inst, pap) && run(mask, x.inst)) {
        g.pap[x.inst] = pap;
        g.alpha[x.inst] = pap > 0.0 ? g.rr[x.inst] / pap : 0.0;
    }
}

// x += alpha p, r -= alpha Ap; r . z of the new residual summed per instance by its last block, which
// counts the iteration, ends the instance's CG solve at the forcing tolerance (floor tol2) and sets
// beta = (r . z)_new / (r . z) and r . z <- (r . z)_new for the direction kernel
__global__ void __launch_bounds__(kNodeBlock) k_cg_step_b(const FomB g, const int* __restrict__ mask, double ic0,
                                                          double tol2) {
    const NodeCtx x = node_ctx(g, mask);
    double s = 0.0;
    if (x.ok) {
        const double alpha = g.alpha[x.inst];
        const double pz = g.minv[x.gn] * ic0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long d = (long long)c * g.NN + x.gn;
            g.cg_x[d] = fma(alpha, g.cg_p[d], g.cg_x[d]);
            const double r = fma(-alpha, g.cg_ap[d], g.cg_r[d]);
            g.cg_r[d] = r;
            s = fma(r * pz, r, s);
        }
    }
    s = block_sum1(s);
    if (threadIdx.x == 0) g.ipart[blockIdx.x] = s;
    double rrn;
    if (last_block_sum(g, x.inst, rrn) && run(mask, x.inst)) {
        const int inst = x.inst;
        g.rrn[inst] = rrn;
        g.istat[2 * inst + 1] += 1;
        if (!(rrn > fmax(tol2, g.cgtol2[inst]) * g.rr0[inst]) || !isfinite(rrn)) g.cgact[inst] = 0;
        const double rr = g.rr[inst];
        g.beta[inst] = rr > 0.0 ? rrn / rr : 0.0;
        g.rr[inst] = rrn;
    }
}

// p = z + beta p
__global__ void __launch_bounds__(kNodeBlock) k_cg_dir_b(const FomB g, const int* __restrict__ mask, double ic0) {
    const NodeCtx x = node_ctx(g, mask);
    if (!x.ok) return;
    const double beta = g.beta[x.inst];
    const double pz = g.minv[x.gn] * ic0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const long long d = (long long)c * g.NN + x.gn;
        g.cg_p[d] = fma(beta, g.cg_p[d], g.cg_r[d] * pz);
    }
}

// u += x on free dofs, refreshed u / h for the force kernel; partials |x|^2 and |u|^2 (free dofs)
__global__ void __launch_bounds__(kNodeBlock) k_imp_update_b(const FomB g, const int* __restrict__ mask) {
    const NodeCtx x = node_ctx(g, mask);
    double sx = 0.0, su = 0.0;
    if (x.ok) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long d = (long long)c * g.NN + x.gn;
            if (is_free(g, x.gn, c)) {
                const double dx = g.cg_x[d];
                const double u = g.u[0][d] + dx;
                g.u[0][d] = u;
                g.us[d] = u * x.I.invh;
                sx = fma(dx, dx, sx);
                su = fma(u, u, su);
            }
        }
    }
    sx = block_sum1(sx);
    su = block_sum1(su);
    if (threadIdx.x == 0) {
        g.ipart[blockIdx.x] = sx;
        g.ipart[g.n_nblk + blockIdx.x] = su;
    }
}

// a = (u - ut) c0, v += dt ((1 - gamma) a_old + gamma a) with gamma = 1/2; Dirichlet / Schwarz data.
// An instance whose Newton solve failed (non-finite residual, or no convergence within the iteration
// cap) gets a non-finite displacement, which the convergence criterion reports.
__global__ void __launch_bounds__(kNodeBlock) k_imp_finish_b(const FomB g, const int* __restrict__ active, int slot1,
                                                             double dt, double c0) {
    const NodeCtx x = node_ctx(g, active);
    if (!x.ok) return;
    if (g.nact[x.inst] != 0) {
#pragma unroll
        for (int c = 0; c < 3; ++c) g.u[0][(long long)c * g.NN + x.gn] = __longlong_as_double(0x7ff8000000000000LL);
        return;
    }
    const uint8_t cm = g.clamp[x.gn];
    const int row = g.srow[x.gn];
    const double* h1 = g.hist + x.I.hist_off + (long long)slot1 * 9 * x.I.ns;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const long long d = (long long)c * g.NN + x.gn;
        if (cm & (1 << c)) {
            g.v[d] = 0.0;
            g.a[d] = 0.0;
        } else if (row >= 0) {
            g.v[d] = h1[(long long)(3 + c) * x.I.ns + row];
            g.a[d] = h1[(long long)(6 + c) * x.I.ns + row];
        } else {
            const double an = c0 * (g.u[0][d] - g.ut[d]);
            g.v[d] = g.v[d] + dt * (0.5 * g.a[d] + 0.5 * an);
            g.a[d] = an;
        }
    }
}

// Device-side loop control (conditional WHILE nodes of a CUDA graph): which = 0 the Newton loop,
// 1 the CG loop.  Entry: reset the loop's counter, enter (Newton) or enter if an instance still has
// a CG solve to do.  Condition at the end of a pass: count the pass, continue while some instance is
// still iterating and the cap is not reached (the loops end after at most max_it passes).
__global__ void k_imp_loop_entry(const FomB g, cudaGraphConditionalHandle h, int which) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    g.iloop[which] = 0;
    unsigned int go = 1;
    if (which == 1) {
        go = 0;
        for (int i = 0; i < g.n_inst; ++i) go |= g.cgact[i] == 1 ? 1u : 0u;
    }
    cudaGraphSetConditional(h, go);
}

__global__ void k_imp_loop_cond(const FomB g, cudaGraphConditionalHandle h, int which, int max_it) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int it = ++g.iloop[which];
    const int* m = which == 0 ? g.nact : g.cgact;
    unsigned int go = 0;
    for (int i = 0; i < g.n_inst; ++i) go |= m[i] == 1 ? 1u : 0u;
    cudaGraphSetConditional(h, (go && it < max_it) ? 1u : 0u);
}

__global__ void k_mask_copy(int n, const int* __restrict__ src, int* dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src ? src[i] : 1;
}

}  // namespace

cudaError_t launch_imp_predict_b(const FomB& g, const int* active, int slot1, double dt, cudaStream_t s) {
    k_imp_predict_b<<<g.n_nblk, kNodeBlock, 0, s>>>(g, active, slot1, dt);
    return cudaGetLastError();
}
cudaError_t launch_imp_residual_b(const FomB& g, const int* mask, double c0, cudaStream_t s) {
    k_imp_residual_b<<<g.n_nblk, kNodeBlock, 0, s>>>(g, mask, c0, 1.0 / c0);   // 1 / c0 once, on the host
    return cudaGetLastError();
}
cudaError_t launch_imp_reduce_b(const FomB& g, const int* mask, int mode, int first, double tol2, cudaStream_t s) {
    k_imp_reduce_b<<<g.n_inst, 128, 0, s>>>(g, mask, mode, first, tol2);
    return cudaGetLastError();
}
cudaError_t launch_cg_ap_b(const FomB& g, const int* mask, double c0, cudaStream_t s) {
    k_cg_ap_b<<<g.n_nblk, kNodeBlock, 0, s>>>(g, mask, c0);
    return cudaGetLastError();
}
cudaError_t launch_cg_step_b(const FomB& g, const int* mask, double c0, double tol2, cudaStream_t s) {
    k_cg_step_b<<<g.n_nblk, kNodeBlock, 0, s>>>(g, mask, 1.0 / c0, tol2);
    return cudaGetLastError();
}
cudaError_t launch_cg_dir_b(const FomB& g, const int* mask, double c0, cudaStream_t s) {
    k_cg_dir_b<<<g.n_nblk, kNodeBlock, 0, s>>>(g, mask, 1.0 / c0);
    return cudaGetLastError();
}
cudaError_t launch_imp_update_b(const FomB& g, const int* mask, cudaStream_t s) {
    k_imp_update_b<<<g.n_nblk, kNodeBlock, 0, s>>>(g, mask);
    return cudaGetLastError();
}
cudaError_t launch_imp_finish_b(const FomB& g, const int* active, int slot1, double dt, double c0, cudaStream_t s) {
    k_imp_finish_b<<<g.n_nblk, kNodeBlock, 0, s>>>(g, active, slot1, dt, c0);
    return cudaGetLastError();
}
cudaError_t launch_imp_loop_entry(const FomB& g, cudaGraphConditionalHandle h, int which, cudaStream_t s) {
    k_imp_loop_entry<<<1, 32, 0, s>>>(g, h, which);
    return cudaGetLastError();
}
cudaError_t launch_imp_loop_cond(const FomB& g, cudaGraphConditionalHandle h, int which, int max_it, cudaStream_t s) {
    k_imp_loop_cond<<<1, 32, 0, s>>>(g, h, which, max_it);
    return cudaGetLastError();
}
cudaError_t launch_mask_copy(int n, const int* src, int* dst, cudaStream_t s) {
    k_mask_copy<<<(n + 127) / 128, 128, 0, s>>>(n, src, dst);
    return cudaGetLastError();
}

}  // namespace osam
