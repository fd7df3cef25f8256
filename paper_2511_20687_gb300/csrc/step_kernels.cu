// Per-step kernels of the O-SAM controller, batched over the instances of a context.
//
// Every kernel takes the group view of one subdomain slot (FomB / RomB) or coupling (CplB) and the
// per-instance `active` mask: instances that have met the convergence criterion of the current
// controller step (Eq. conv_criterion) are skipped, so each instance performs exactly the
// iterations it would perform alone.  Blocks never span two instances.
//   FOM: hex8 force (Sec. 2 / Appendix A, sum-factorised, hex8_math.cuh), corrector + predictor of
//        the explicit Newmark scheme (beta = 0, gamma = 1/2) with Dirichlet and Schwarz data,
//        state save / restore, criterion partial sums, trace Pi(u, v, a) at a neighbour's Schwarz
//        nodes, publication into the neighbour's history, zero-order hold.
//   ROM: boundary projection ghat = Phi_S^T s, reduced step qdd = K q + H kron_c(q) + B ghat + c,
//        reconstruction (Pi Phi_rows) q, criterion partial sums, save / restore.
//   Controller: per-instance criterion and convergence flags; the last block sets the condition of
//        the CUDA graph's while node (any instance still iterating).
#include <cuda_runtime.h>

#include <cstdint>

#include "hex8_math.cuh"
#include "osam_internal.h"
#include "trace_item.cuh"

namespace osam {

namespace {

using namespace hex8;

constexpr int kRomBlock = 128;   // columns per block of the reduced step
constexpr int kRomRows = 8;      // rows per block of the reduced step
constexpr int kMaxR = 256;

// ------------------------------------------------------------------------------------------------
// FOM
// ------------------------------------------------------------------------------------------------
template <int MAT, typename T, int MODE>
__device__ __forceinline__ void force_body(const FomB& g, const int* __restrict__ active, const TraceFuse& tr) {
    if ((int)blockIdx.x >= g.n_eblk) {
        trace::fused_trace_block(tr, active, g, (int)blockIdx.x - g.n_eblk);
        return;
    }
    const int2 b = g.eblk[blockIdx.x];
    if (active && !active[b.x]) return;
    const InstFom I = g.inst[b.x];
    const int e = b.y + threadIdx.x;
    if (e >= I.ne) return;
    const int i = e % I.nx;
    const int t = e / I.nx;
    const int j = t % I.ny;
    const int k = t / I.ny;
    const int sy = I.nx + 1, sz = (I.nx + 1) * (I.ny + 1);
    const int n0 = i + sy * j + sz * k;
    int node[8];
#pragma unroll
    for (int c8 = 0; c8 < 8; ++c8) node[c8] = n0 + (c8 & 1) + ((c8 >> 1) & 1) * sy + ((c8 >> 2) & 1) * sz;
    T m1, m2, m3;
    if (I.lam_e || I.mu_e)
        material_factors<MAT, T>(I.lam_e ? I.lam_e[e] : I.lam, I.mu_e ? I.mu_e[e] : I.mu, I.wq, I.wq3, m1, m2, m3);
    else { m1 = T(I.m1); m2 = T(I.m2); m3 = T(I.m3); }
    T Dx[3][2][2], Dy[3][2][2], Dz[3][2][2];
    if constexpr (sizeof(T) == 4) {
        // FP32 force: differences of the float split of u/h (the node kernel writes it beside u/h)
        const float2* ub2 = g.u2 + I.node_off;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float2 U2[8];
#pragma unroll
            for (int c8 = 0; c8 < 8; ++c8) U2[c8] = ub2[(long long)c * g.NN + node[c8]];
            edge_differences_split(U2, Dx[c], Dy[c], Dz[c]);
        }
    } else {
        const double* ub = g.us + I.node_off;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double U[8];
#pragma unroll
            for (int c8 = 0; c8 < 8; ++c8) U[c8] = ub[(long long)c * g.NN + node[c8]];
            edge_differences_prescaled<T>(U, Dx[c], Dy[c], Dz[c]);
        }
    }
    T F[3][8];
    element_force<MAT, T>(Dx, Dy, Dz, m1, m2, m3, F);
    if (MODE == kAtomic) {
        T* f = static_cast<T*>(g.f) + I.node_off;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int c8 = 0; c8 < 8; ++c8) atomic_add(f + (long long)c * g.NN + node[c8], F[c][c8]);
    } else {
        T* fe = static_cast<T*>(g.fe) + I.elem_off;
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8)
#pragma unroll
            for (int c = 0; c < 3; ++c) fe[(long long)(c8 * 3 + c) * g.NE + e] = F[c][c8];
    }
}

// Tiled FP64 force: one block of 128 threads per 8x4x4 tile of elements.  The edge differences and
// the first interpolation stage of the gradients are shared by neighbouring elements (an x-edge pair
// interpolated along y serves the elements below and above it, and every edge difference serves two
// such pairs), so the block computes them once per tile in shared memory and each thread finishes its
// element with the second stage.  The arithmetic per value is the one of edge_differences_prescaled +
// lerp2, so the result equals the untiled kernel's bit for bit; the sharing saves ~43 of the ~780 FP64
// operations per element.
constexpr int kTX = 8, kTY = 4, kTZ = 4;

template <int MAT, int MODE>
__device__ __forceinline__ void force_tile_body(const FomB& g, const int* __restrict__ active, const TraceFuse& tr) {
    if ((int)blockIdx.x >= g.n_tblk) {
        trace::fused_trace_block(tr, active, g, (int)blockIdx.x - g.n_tblk);
        return;
    }
    __shared__ double su[3][kTZ + 1][kTY + 1][kTX + 1];  // u / h at the tile's nodes
    __shared__ double sdx[3][kTZ + 1][kTY + 1][kTX];     // x-edge differences [c][k][j][i]
    __shared__ double sdy[3][kTZ + 1][kTY][kTX + 1];     // y-edge differences
    __shared__ double sdz[3][kTZ][kTY + 1][kTX + 1];     // z-edge differences
    __shared__ double sax[3][kTZ + 1][kTY][kTX][2];     // x-edges interpolated along y: [c][k][j][i][gy]
    __shared__ double say[3][kTZ + 1][kTY][kTX][2];     // y-edges interpolated along x: [c][k][j][i][gx]
    __shared__ double saz[3][kTZ][kTY + 1][kTX][2];     // z-edges interpolated along x: [c][k][j][i][gx]
    const int4 tb = g.tblk[blockIdx.x];
    if (active && !active[tb.x]) return;
    const InstFom I = g.inst[tb.x];
    const int i0 = tb.y, j0 = tb.z, k0 = tb.w;
    const int tid = threadIdx.x;
    const int sy = I.nx + 1, sz = (I.nx + 1) * (I.ny + 1);
    // (1) nodal values of the tile (zero beyond the mesh; only elements inside read them)
    for (int q = tid; q < 3 * (kTZ + 1) * (kTY + 1) * (kTX + 1); q += blockDim.x) {
        const int c = q / ((kTZ + 1) * (kTY + 1) * (kTX + 1));
        const int rem = q % ((kTZ + 1) * (kTY + 1) * (kTX + 1));
        const int kk = rem / ((kTY + 1) * (kTX + 1)), jj = (rem / (kTX + 1)) % (kTY + 1), ii = rem % (kTX + 1);
        const int gi = i0 + ii, gj = j0 + jj, gk = k0 + kk;
        double v = 0.0;
        if (gi <= I.nx && gj <= I.ny && gk <= I.nz)
            v = g.us[(long long)c * g.NN + I.node_off + gi + (long long)sy * gj + (long long)sz * gk];
        su[c][kk][jj][ii] = v;
    }
    __syncthreads();
    // (2) edge differences, each once per tile (two staged pairs share every one of them)
    constexpr int nX = (kTZ + 1) * (kTY + 1) * kTX, nY = (kTZ + 1) * kTY * (kTX + 1), nZ = kTZ * (kTY + 1) * (kTX + 1);
    for (int q = tid; q < 3 * (nX + nY + nZ); q += blockDim.x) {
        const int c = q / (nX + nY + nZ), w = q % (nX + nY + nZ);
        if (w < nX) {
            const int k = w / ((kTY + 1) * kTX), j = (w / kTX) % (kTY + 1), i = w % kTX;
            sdx[c][k][j][i] = su[c][k][j][i + 1] - su[c][k][j][i];
        } else if (w < nX + nY) {
            const int v = w - nX, k = v / (kTY * (kTX + 1)), j = (v / (kTX + 1)) % kTY, i = v % (kTX + 1);
            sdy[c][k][j][i] = su[c][k][j + 1][i] - su[c][k][j][i];
        } else {
            const int v = w - nX - nY, k = v / ((kTY + 1) * (kTX + 1)), j = (v / (kTX + 1)) % (kTY + 1),
                      i = v % (kTX + 1);
            sdz[c][k][j][i] = su[c][k + 1][j][i] - su[c][k][j][i];
        }
    }
    __syncthreads();
    // (3) the first interpolation stage, 3 directions x 3 components x 160 pairs
    const double G[2] = {hex8::kG0, hex8::kG1};
    for (int q = tid; q < 3 * 3 * 160; q += blockDim.x) {
        const int dir = q / 480, c = (q / 160) % 3, w = q % 160;
        // Neo-Hookean: the derivative of component c along direction c gets the 1 of F's diagonal here
        // (once per staged pair instead of once per Gauss point), as element_force does in lerp2
        const bool diag = MAT == OSAM_NEO_HOOKEAN && c == dir;
        if (dir == 0) {          // x-edges (i; j, k) and (i; j + 1, k), interpolated along y
            const int k = w / 32, j = (w / 8) % 4, i = w % 8;
            const double d0 = sdx[c][k][j][i], d1 = sdx[c][k][j + 1][i];
            const double dd = d1 - d0, base = diag ? d0 + 1.0 : d0;
            sax[c][k][j][i][0] = hex8::fmaT(G[0], dd, base);
            sax[c][k][j][i][1] = hex8::fmaT(G[1], dd, base);
        } else if (dir == 1) {   // y-edges (i, j; k) and (i + 1, j; k), interpolated along x
            const int k = w / 32, j = (w / 8) % 4, i = w % 8;
            const double d0 = sdy[c][k][j][i], d1 = sdy[c][k][j][i + 1];
            const double dd = d1 - d0, base = diag ? d0 + 1.0 : d0;
            say[c][k][j][i][0] = hex8::fmaT(G[0], dd, base);
            say[c][k][j][i][1] = hex8::fmaT(G[1], dd, base);
        } else {                 // z-edges (i, j, k) and (i + 1, j, k), interpolated along x
            const int k = w / 40, j = (w / 8) % 5, i = w % 8;
            const double d0 = sdz[c][k][j][i], d1 = sdz[c][k][j][i + 1];
            const double dd = d1 - d0, base = diag ? d0 + 1.0 : d0;
            saz[c][k][j][i][0] = hex8::fmaT(G[0], dd, base);
            saz[c][k][j][i][1] = hex8::fmaT(G[1], dd, base);
        }
    }
    __syncthreads();
    // (4) one element per thread: second stage, constitutive law, transposed interpolation
    const int ti = tid % kTX, tj = (tid / kTX) % kTY, tk = tid / (kTX * kTY);
    const int ei = i0 + ti, ej = j0 + tj, ek = k0 + tk;
    if (ei >= I.nx || ej >= I.ny || ek >= I.nz) return;
    const int e = ei + I.nx * (ej + I.ny * ek);
    double Gx[3][2][2], Gy[3][2][2], Gz[3][2][2];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            double e0 = sax[c][tk][tj][ti][a], d = sax[c][tk + 1][tj][ti][a] - e0;   // along z
            Gx[c][a][0] = hex8::fmaT(G[0], d, e0);
            Gx[c][a][1] = hex8::fmaT(G[1], d, e0);
            e0 = say[c][tk][tj][ti][a];
            d = say[c][tk + 1][tj][ti][a] - e0;                                       // along z
            Gy[c][a][0] = hex8::fmaT(G[0], d, e0);
            Gy[c][a][1] = hex8::fmaT(G[1], d, e0);
            e0 = saz[c][tk][tj][ti][a];
            d = saz[c][tk][tj + 1][ti][a] - e0;                                       // along y
            Gz[c][a][0] = hex8::fmaT(G[0], d, e0);
            Gz[c][a][1] = hex8::fmaT(G[1], d, e0);
        }
    double m1, m2, m3;
    if (I.lam_e || I.mu_e)
        material_factors<MAT, double>(I.lam_e ? I.lam_e[e] : I.lam, I.mu_e ? I.mu_e[e] : I.mu, I.wq, I.wq3, m1, m2,
                                      m3);
    else { m1 = I.m1; m2 = I.m2; m3 = I.m3; }
    double F[3][8];
    element_force_grad<MAT, double>(Gx, Gy, Gz, m1, m2, m3, F);
    if (MODE == kAtomic) {
        double* f = static_cast<double*>(g.f) + I.node_off;
        const int n0 = ei + sy * ej + sz * ek;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int c8 = 0; c8 < 8; ++c8)
                atomic_add(f + (long long)c * g.NN + n0 + (c8 & 1) + ((c8 >> 1) & 1) * sy + ((c8 >> 2) & 1) * sz,
                           F[c][c8]);
    } else {
        double* fe = static_cast<double*>(g.fe) + I.elem_off;
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8)
#pragma unroll
            for (int c = 0; c < 3; ++c) fe[(long long)(c8 * 3 + c) * g.NE + e] = F[c][c8];
    }
}

// the tiled force as compiled for its natural register count (166 for Neo-Hookean: 3 blocks per SM)
// and capped at 128 registers (4 blocks per SM, a few spilled values): 1000 tiles of the 40x40x80
// mesh are 2.19 waves of the first and 1.64 of the second; the autotuner times both
template <int MAT, int MODE>
__global__ void __launch_bounds__(128) k_force_tile_b(const FomB g, const int* __restrict__ active,
                                                      const TraceFuse tr) {
    force_tile_body<MAT, MODE>(g, active, tr);
}

template <int MAT>
__global__ void __launch_bounds__(128, 4) k_force_tile_occ_b(const FomB g, const int* __restrict__ active,
                                                             const TraceFuse tr) {
    force_tile_body<MAT, kGather>(g, active, tr);
}

// the force kernel at its natural register count (168 for Neo-Hookean FP64: 12 warps per SM) ...
template <int MAT, typename T, int MODE>
__global__ void __launch_bounds__(256) k_force_b(const FomB g, const int* __restrict__ active, const TraceFuse tr) {
    force_body<MAT, T, MODE>(g, active, tr);
}

// ... and capped at 128 registers (16 warps per SM, a few spilled values): the autotuner keeps
// whichever is faster on the problem at hand
template <int MAT>
__global__ void __launch_bounds__(128, 4) k_force_occ_b(const FomB g, const int* __restrict__ active,
                                                        const TraceFuse tr) {
    force_body<MAT, double, kGather>(g, active, tr);
}

// us = u[0] / h (input of the FP64 force at the start of an interval / after a state change)
__global__ void __launch_bounds__(kNodeBlock) k_scale_u0_b(const FomB g, const int* __restrict__ active) {
    const int2 b = g.nblk[blockIdx.x];
    if (active && !active[b.x]) return;
    const InstFom I = g.inst[b.x];
    const int n = b.y + threadIdx.x;
    if (n >= I.nn) return;
    const long long gn = I.node_off + n;
#pragma unroll
    for (int c = 0; c < 3; ++c) g.us[(long long)c * g.NN + gn] = g.u[0][(long long)c * g.NN + gn] * I.invh;
}

// a = -M^-1 f on every non-clamped dof from the FP64 element buffer (initial acceleration)
__global__ void __launch_bounds__(kNodeBlock) k_init_accel_b(const FomB g, const int* __restrict__ active) {
    const int2 b = g.nblk[blockIdx.x];
    if (active && !active[b.x]) return;
    const InstFom I = g.inst[b.x];
    const int n = b.y + threadIdx.x;
    if (n >= I.nn) return;
    const int i = n % (I.nx + 1);
    const int t = n / (I.nx + 1);
    const int j = t % (I.ny + 1);
    const int k = t / (I.ny + 1);
    const long long gn = I.node_off + n;
    const uint8_t cm = g.clamp[gn];
    const double* fe = static_cast<const double*>(g.fe) + I.elem_off;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double f = gather_force<double>(fe, I.nx, I.ny, I.nz, (int)g.NE, i, j, k, c);
        g.a[(long long)c * g.NN + gn] = (cm & (1 << c)) ? 0.0 : -f * g.minv[gn];
    }
}

// Corrector of substep j and predictor of substep j+1 (explicit Newmark beta = 0, gamma = 1/2):
//   free dofs:  a' = -f/m;  v += dt/2 (a + a');  a = a';  u^{j+2} = u^{j+1} + dt v + dt^2/2 a
//   clamped:    u = v = a = 0
//   Schwarz:    v, a from history slot j+1 (slot1); u^{j+2} from history slot j+2 (slot2)
// predict_only: write the predictor of ucur with the current (v, a) (start of an interval).
template <typename TF, int MODE>
__global__ void __launch_bounds__(kNodeBlock) k_node_b(const FomB g, const int* __restrict__ active, int slot1,
                                                      int slot2, int predict_only, const double* ucur, double* unext,
                                                      double dt) {
    const int2 b = g.nblk[blockIdx.x];
    if (active && !active[b.x]) return;
    const InstFom I = g.inst[b.x];
    const int n = b.y + threadIdx.x;
    if (n >= I.nn) return;
    const int i = n % (I.nx + 1);
    const int t = n / (I.nx + 1);
    const int j = t % (I.ny + 1);
    const int k = t / (I.ny + 1);
    const long long gn = I.node_off + n;
    const uint8_t cm = g.clamp[gn];
    const int row = g.srow[gn];
    const double hdt = 0.5 * dt, hdt2 = 0.5 * dt * dt;
    const double minv = g.minv[gn];
    const double* h1 = slot1 >= 0 ? g.hist + I.hist_off + (long long)slot1 * 9 * I.ns : nullptr;
    const double* h2 = slot2 >= 0 ? g.hist + I.hist_off + (long long)slot2 * 9 * I.ns : nullptr;
    const TF* fe = static_cast<const TF*>(g.fe) + I.elem_off;
    TF* fa = static_cast<TF*>(g.f);
    // all loads of a free node first (state and the element contributions of the three components,
    // summed per component in the fixed corner order), so that they are in flight together
    double uc[3], vc[3], ac[3], f[3] = {0.0, 0.0, 0.0};
    TF fs[3] = {TF(0), TF(0), TF(0)};   // the gather sums in the element buffer's precision
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const long long d = (long long)c * g.NN + gn;
        uc[c] = ucur[d];
        vc[c] = g.v[d];
        ac[c] = g.a[d];
    }
    if (!predict_only && row < 0 && cm != 7) {
        if (MODE == kGather) {
#pragma unroll
            for (int az = 0; az < 2; ++az) {
                const int ke = k - az;
                if (ke < 0 || ke >= I.nz) continue;
#pragma unroll
                for (int ay = 0; ay < 2; ++ay) {
                    const int je = j - ay;
                    if (je < 0 || je >= I.ny) continue;
#pragma unroll
                    for (int ax = 0; ax < 2; ++ax) {
                        const int ie = i - ax;
                        if (ie < 0 || ie >= I.nx) continue;
                        const long long e = ie + (long long)I.nx * (je + I.ny * ke);
                        const int corner = ax + 2 * ay + 4 * az;
#pragma unroll
                        for (int c = 0; c < 3; ++c) fs[c] += __ldg(fe + (long long)(corner * 3 + c) * g.NE + e);
                    }
                }
            }
            // FP64: the same sums; FP32 force: summed in FP32 (its own precision) and widened once, by
            // integer operations (f64_of: exact)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if constexpr (sizeof(TF) == 4) f[c] = f64_of(fs[c]);
                else f[c] = fs[c];
            }
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if constexpr (sizeof(TF) == 4) f[c] = f64_of(fa[(long long)c * g.NN + gn]);
                else f[c] = fa[(long long)c * g.NN + gn];
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const long long d = (long long)c * g.NN + gn;
        double un;
        if (cm & (1 << c)) {
            g.v[d] = 0.0;
            g.a[d] = 0.0;
            un = 0.0;
            if (MODE == kAtomic && !predict_only) fa[d] = TF(0);
        } else if (row >= 0) {
            if (!predict_only) {
                g.v[d] = h1[(long long)(3 + c) * I.ns + row];
                g.a[d] = h1[(long long)(6 + c) * I.ns + row];
                if (MODE == kAtomic) fa[d] = TF(0);
            }
            un = h2 ? h2[(long long)c * I.ns + row] : 0.0;
        } else {
            double vn = vc[c], an = ac[c];
            if (!predict_only) {
                if (MODE == kAtomic) fa[d] = TF(0);
                const double anew = -f[c] * minv;
                vn = fma(hdt, an + anew, vn);
                an = anew;
                g.v[d] = vn;
                g.a[d] = an;
            }
            un = fma(hdt2, an, fma(dt, vn, uc[c]));
        }
        if (h2) {
            unext[d] = un;
            g.us[d] = un * I.invh;
            if (sizeof(TF) == 4) g.u2[d] = split_f2(un * I.invh);   // FP32 force input
        }
    }
}

// save (restore = 0) or restore (restore = 1) the state at the start of the controller interval
__global__ void __launch_bounds__(kNodeBlock) k_saverest_fom_b(const FomB g, const int* __restrict__ active,
                                                              int restore) {
    const int2 b = g.nblk[blockIdx.x];
    if (active && !active[b.x]) return;
    const InstFom I = g.inst[b.x];
    const int n = b.y + threadIdx.x;
    if (n >= I.nn) return;
    const long long gn = I.node_off + n;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const long long d = (long long)c * g.NN + gn;
        if (restore) { g.u[0][d] = g.su[d]; g.v[d] = g.sv[d]; g.a[d] = g.sa[d]; }
        else { g.su[d] = g.u[0][d]; g.sv[d] = g.v[d]; g.sa[d] = g.a[d]; }
    }
}

// u[0] <- u[1] (an interval with an odd substep count ends in the second displacement buffer)
__global__ void __launch_bounds__(kNodeBlock) k_copy_u10_b(const FomB g, const int* __restrict__ active) {
    const int2 b = g.nblk[blockIdx.x];
    if (active && !active[b.x]) return;
    const InstFom I = g.inst[b.x];
    const int n = b.y + threadIdx.x;
    if (n >= I.nn) return;
    const long long gn = I.node_off + n;
#pragma unroll
    for (int c = 0; c < 3; ++c) g.u[0][(long long)c * g.NN + gn] = g.u[1][(long long)c * g.NN + gn];
}

__device__ __forceinline__ void block_sum2(double& x, double& y) {
    __shared__ double sx[32], sy[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_down_sync(0xffffffffu, x, o);
        y += __shfl_down_sync(0xffffffffu, y, o);
    }
    const int w = threadIdx.x / 32, l = threadIdx.x % 32;
    const int nw = (blockDim.x + 31) / 32;
    __syncthreads();
    if (l == 0) { sx[w] = x; sy[w] = y; }
    __syncthreads();
    if (w == 0) {
        x = l < nw ? sx[l] : 0.0;
        y = l < nw ? sy[l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_down_sync(0xffffffffu, x, o);
            y += __shfl_down_sync(0xffffffffu, y, o);
        }
    }
}

// criterion partial sums over free dofs of one node block; remembers the iterate
__global__ void __launch_bounds__(kNodeBlock) k_norms_fom_b(const FomB g, const int* __restrict__ active, double dt) {
    const int2 b = g.nblk[blockIdx.x];
    if (active && !active[b.x]) return;
    const InstFom I = g.inst[b.x];
    const int n = b.y + threadIdx.x;
    double num = 0.0, den = 0.0;
    if (n < I.nn) {
        const long long gn = I.node_off + n;
        const uint8_t cm = g.clamp[gn];
        const bool sch = g.srow[gn] >= 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long d = (long long)c * g.NN + gn;
            const double un = g.u[0][d], vn = g.v[d];
            if (!(cm & (1 << c)) && !sch) {
                const double x = (un - g.pu[d]) + dt * (vn - g.pv[d]);
                const double y = fma(dt, vn, un);
                num = fma(x, x, num);
                den = fma(y, y, den);
            }
            g.pu[d] = un;
            g.pv[d] = vn;
        }
    }
    block_sum2(num, den);
    if (threadIdx.x == 0) {
        g.partial[2 * blockIdx.x] = num;
        g.partial[2 * blockIdx.x + 1] = den;
    }
}

__device__ __forceinline__ long long dst_index(const CplB& c, int inst, int slot, int f, int cc, int row) {
    const int nd = c.dst_nd[inst];
    const long long base = c.dst_hist_off[inst];
    return c.dst_rom ? base + (long long)(slot * 3 + f) * nd + 3 * row + cc
                     : base + (long long)((slot * 3 + f) * 3 + cc) * nd + row;
}

// trace of a FOM source at slot `slot`: rec[inst][slot][f][c][row] = sum_b w_b field_f,c[donor_b]
__global__ void k_trace_b(const CplB c, const int* __restrict__ active, const FomB src, const double* u, int slot) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < 3 * c.R) trace::trace_item(c, active, src, u, slot, t);
}
// temporal interpolant Xi (Sec. 4.1): destination level m of nd (time m T / nd) lies at source level
// l + w of ns (time (l + w) T / ns); w = 0 exactly when the levels coincide
__device__ __forceinline__ int xi_level(int m, int ns, int nd, double& w) {
    const long long num = (long long)m * ns;
    const int l = (int)(num / nd);
    const long long rem = num - (long long)l * nd;
    w = rem ? (double)rem / (double)nd : 0.0;
    return l;
}

// publish a FOM source's recorded trace (levels 0..ns) into destination levels [slot0, slot0 + nslots)
// of nd, linear in time between the bracketing source levels
__global__ void k_publish_b(const CplB c, const int* __restrict__ active, int slot0, int nslots, int ns, int nd) {
    const long long total = (long long)c.R * 9 * nslots;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= total) return;
    const int gr = (int)(t % c.R);
    const long long q = t / c.R;
    const int fc = (int)(q % 9);
    const int slot = slot0 + (int)(q / 9);
    const int inst = c.rinst[gr];
    if (active && !active[inst]) return;
    const int li = gr - c.row_first[inst], nr = c.nrow[inst];
    double w;
    const int l = xi_level(slot, ns, nd, w);
    const double* rec = c.rec + c.rec_off[inst];
    double val = rec[((long long)l * 9 + fc) * nr + li];
    if (w != 0.0) val = (1.0 - w) * val + w * rec[((long long)(l + 1) * 9 + fc) * nr + li];
    c.dst_hist[dst_index(c, inst, slot, fc / 3, fc % 3, c.row[gr])] = val;
}

// zero-order hold of a FOM source's current state into every slot of the destination history and
// into level 0 of the recorded trace (the state at the start of the interval)
__global__ void k_zoh_fom_b(const CplB c, const int* __restrict__ active, const FomB src, int nslots) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * c.R) return;
    const int gr = t / 3, cc = t % 3;
    const int inst = c.rinst[gr];
    if (active && !active[inst]) return;
    double s[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const double w = c.dw[8 * gr + b];
        const long long d = (long long)cc * src.NN + c.dnode[8 * gr + b];
        s[0] = fma(w, src.u[0][d], s[0]);
        s[1] = fma(w, src.v[d], s[1]);
        s[2] = fma(w, src.a[d], s[2]);
    }
    for (int slot = 0; slot < nslots; ++slot)
#pragma unroll
        for (int f = 0; f < 3; ++f) c.dst_hist[dst_index(c, inst, slot, f, cc, c.row[gr])] = s[f];
    const int li = gr - c.row_first[inst], nr = c.nrow[inst];
#pragma unroll
    for (int f = 0; f < 3; ++f) c.rec[c.rec_off[inst] + (long long)(3 * f + cc) * nr + li] = s[f];
}

// ------------------------------------------------------------------------------------------------
// ROM
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double x) {
    __shared__ double s[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    const int w = threadIdx.x / 32, l = threadIdx.x % 32;
    __syncthreads();
    if (l == 0) s[w] = x;
    __syncthreads();
    const int nw = (blockDim.x + 31) / 32;
    if (w == 0) {
        x = l < nw ? s[l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    }
    return x;  // valid in thread 0
}

__global__ void k_rom_record0_b(const RomB r, const int* __restrict__ active) {
    const int inst = blockIdx.x;
    if (active && !active[inst]) return;
    const InstRom I = r.inst[inst];
    for (int k = threadIdx.x; k < 3 * I.r; k += blockDim.x) r.qrec[I.qrec_off + k] = r.q[I.q_off + k];
}

// ghat[slot][k] = sum_m PhiSt[k][m] hist[slot][u][m]; one block per (k, slot, instance)
__global__ void k_rom_project_b(const RomB r, const int* __restrict__ active, int slot0) {
    const int inst = blockIdx.z;
    if (active && !active[inst]) return;
    const InstRom I = r.inst[inst];
    const int k = blockIdx.x;
    if (k >= I.rs) return;
    const int slot = slot0 + blockIdx.y;
    const double* s = r.hist + I.hist_off + (long long)slot * 3 * I.nsdof;
    const double* p = r.PhiSt + I.PhiSt_off + (long long)k * I.nsdof;
    double acc = 0.0;
    for (int m = threadIdx.x; m < I.nsdof; m += blockDim.x) acc = fma(p[m], s[m], acc);
    acc = block_sum(acc);
    if (threadIdx.x == 0) r.ghat[I.ghat_off + (long long)slot * I.rs + k] = acc;
}

// Column-split GEMV of the packed operator with phi = [q, kron_c(q), ghat, 1] at the predicted q;
// the last block of each instance reduces the partial sums in a fixed order and applies the
// corrector (rhs_only: qdd = rhs(q) without time stepping).
__global__ void __launch_bounds__(kRomBlock) k_rom_step_b(const RomB r, const int* __restrict__ active, int slot,
                                                          double dt, int rhs_only) {
    __shared__ double qp[kMaxR];
    __shared__ double red[kRomBlock / 32][kRomRows];
    __shared__ bool last_block;
    const int inst = blockIdx.z;
    if (active && !active[inst]) return;
    const InstRom I = r.inst[inst];
    if ((int)blockIdx.x >= I.gx || (int)blockIdx.y >= I.gy) return;
    const int tid = threadIdx.x;
    double* q = r.q + I.q_off;
    for (int t = tid; t < I.r; t += blockDim.x) {
        const double qv = q[t];
        qp[t] = rhs_only ? qv : fma(0.5 * dt * dt, q[2 * I.r + t], fma(dt, q[I.r + t], qv));
    }
    __syncthreads();
    const int col = blockIdx.x * kRomBlock + tid;
    double phi = 0.0;
    if (col < I.r) phi = qp[col];
    else if (col < I.r + I.nq) { const short2 ij = r.kij[I.kij_off + col - I.r]; phi = qp[ij.x] * qp[ij.y]; }
    else if (col < I.r + I.nq + I.nc) {
        const short4 t3 = r.kijk[I.kijk_off + col - I.r - I.nq];
        phi = qp[t3.x] * qp[t3.y] * qp[t3.z];
    }
    else if (col < I.r + I.nq + I.nc + I.rs) phi = r.ghat[I.ghat_off + (long long)slot * I.rs + col - I.r - I.nq - I.nc];
    else if (col == I.d - 1) phi = 1.0;
    const double* O = r.O + I.O_off;
    double part[kRomRows];
#pragma unroll
    for (int rr = 0; rr < kRomRows; ++rr) {
        const int row = blockIdx.y * kRomRows + rr;
        part[rr] = (row < I.r && col < I.d) ? O[(long long)row * I.d + col] * phi : 0.0;
    }
#pragma unroll
    for (int rr = 0; rr < kRomRows; ++rr)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part[rr] += __shfl_down_sync(0xffffffffu, part[rr], o);
    if (tid % 32 == 0)
#pragma unroll
        for (int rr = 0; rr < kRomRows; ++rr) red[tid / 32][rr] = part[rr];
    __syncthreads();
    double* partial = r.partial + I.partial_off;
    if (tid < kRomRows) {
        const int row = blockIdx.y * kRomRows + tid;
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < kRomBlock / 32; ++w) s += red[w][tid];
        if (row < I.r) partial[(long long)blockIdx.x * I.r + row] = s;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const unsigned int ticket = atomicAdd(r.counter + inst, 1u);
        last_block = ticket == (unsigned int)(I.gx * I.gy - 1);
    }
    __syncthreads();
    if (!last_block) return;
    __threadfence();
    double* rec = rhs_only ? nullptr : r.qrec + I.qrec_off + (long long)slot * 3 * I.r;
    for (int row = tid; row < I.r; row += blockDim.x) {
        double acc = 0.0;
        for (int bx = 0; bx < I.gx; ++bx) acc += __ldcg(partial + (long long)bx * I.r + row);
        if (rhs_only) {
            q[2 * I.r + row] = acc;
        } else {
            const double qd = fma(0.5 * dt, q[2 * I.r + row] + acc, q[I.r + row]);
            q[row] = qp[row];
            q[I.r + row] = qd;
            q[2 * I.r + row] = acc;
            rec[row] = qp[row];
            rec[I.r + row] = qd;
            rec[2 * I.r + row] = acc;
        }
    }
    if (tid == 0) r.counter[inst] = 0u;
}

// s_dst[slot][f][3 i + c] = sum_k Rt[k][3 i + c] q_src(t_slot)[f][k]; grid (columns, slots, fields).
// q_src(t_slot) is the recorded source level, or linear in time between the two bracketing source
// levels (temporal interpolant Xi) when the substep counts differ; zoh: the current state.
__global__ void k_rom_reconstruct_b(const CplB c, const int* __restrict__ active, const RomB src, int zoh, int slot0,
                                    int ns, int nd) {
    const int gc = blockIdx.x * blockDim.x + threadIdx.x;
    if (gc >= 3 * c.R) return;
    const int gr = gc / 3, cc = gc % 3;
    const int inst = c.rinst[gr];
    if (active && !active[inst]) return;
    const InstRom I = src.inst[inst];
    const int li = gr - c.row_first[inst], nr = c.nrow[inst];
    const int slot = slot0 + blockIdx.y;
    const int f = blockIdx.z;
    double w = 0.0;
    const int l = zoh ? 0 : xi_level(slot, ns, nd, w);
    const double* q = zoh ? src.q + I.q_off + (long long)f * I.r
                          : src.qrec + I.qrec_off + ((long long)l * 3 + f) * I.r;
    const double* Rt = c.Rt + c.Rt_off[inst];
    const int col = 3 * li + cc;
    double acc = 0.0;
    if (w == 0.0) {
        for (int k = 0; k < I.r; ++k) acc = fma(Rt[(long long)k * 3 * nr + col], q[k], acc);
    } else {
        const double* q1 = q + 3LL * I.r;
        for (int k = 0; k < I.r; ++k) acc = fma(Rt[(long long)k * 3 * nr + col], (1.0 - w) * q[k] + w * q1[k], acc);
    }
    c.dst_hist[dst_index(c, inst, slot, f, cc, c.row[gr])] = acc;
}

__global__ void k_rom_norms_b(const RomB r, const int* __restrict__ active, double dt) {
    const int inst = blockIdx.x;
    if (active && !active[inst]) return;
    const InstRom I = r.inst[inst];
    const double* q = r.q + I.q_off;
    double* pq = r.pq + I.q_off;
    double num = 0.0, den = 0.0;
    for (int k = threadIdx.x; k < I.r; k += blockDim.x) {
        const double x = (q[k] - pq[k]) + dt * (q[I.r + k] - pq[I.r + k]);
        const double y = fma(dt, q[I.r + k], q[k]);
        num = fma(x, x, num);
        den = fma(y, y, den);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < I.r; k += blockDim.x) {
        pq[k] = q[k];
        pq[I.r + k] = q[I.r + k];
    }
    block_sum2(num, den);
    if (threadIdx.x == 0) {
        r.npart[2 * inst] = num;
        r.npart[2 * inst + 1] = den;
    }
}

__global__ void k_saverest_rom_b(const RomB r, const int* __restrict__ active, int restore) {
    const int inst = blockIdx.x;
    if (active && !active[inst]) return;
    const InstRom I = r.inst[inst];
    for (int k = threadIdx.x; k < 3 * I.r; k += blockDim.x) {
        if (restore) r.q[I.q_off + k] = r.sq[I.q_off + k];
        else r.sq[I.q_off + k] = r.q[I.q_off + k];
    }
}

// ------------------------------------------------------------------------------------------------
// controller
// ------------------------------------------------------------------------------------------------
__global__ void k_reset_ctl(const CtlB c) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.n_inst) return;
    c.active[i] = 1;
    c.iters[i] = 0;
    c.status[i] = OSAM_OK;
    c.cnum[i] = 0.0;
    c.cden[i] = 0.0;
    if (i == 0) *c.any_active = 1;
}

// one block per instance: criterion sums (fixed order), convergence decision; the last block to
// finish publishes "any instance still iterating" (and sets the while-node condition in a graph)
__global__ void __launch_bounds__(256) k_controller(const CtlB c, cudaGraphConditionalHandle h, int use_cond) {
    __shared__ bool last_block;
    const int inst = blockIdx.x;
    const bool act = c.active[inst] != 0;
    double num = 0.0, den = 0.0;
    if (act) {
        for (int s = 0; s < c.n_fom; ++s) {
            const int b0 = c.fom_blk_off[s][inst], b1 = c.fom_blk_off[s][inst + 1];
            for (int b = b0 + (int)threadIdx.x; b < b1; b += blockDim.x) {
                num += c.fom_partial[s][2 * b];
                den += c.fom_partial[s][2 * b + 1];
            }
        }
    }
    block_sum2(num, den);
    if (threadIdx.x == 0 && act) {
        for (int s = 0; s < c.n_rom; ++s) {
            num += c.rom_npart[s][2 * inst];
            den += c.rom_npart[s][2 * inst + 1];
        }
        const int n = c.iters[inst] + 1;
        c.iters[inst] = n;
        c.cnum[inst] = num;
        c.cden[inst] = den;
        int done = 0, st = OSAM_OK;
        if (!(isfinite(num) && isfinite(den))) { done = 1; st = OSAM_ENONFINITE; }
        else if (c.ncpl == 0) done = 1;
        else if (n >= 2 && (num < c.tol_abs2 || num < c.tol_rel2 * den)) done = 1;
        else if (n >= c.max_it) { done = 1; st = OSAM_MAXITER; }
        if (done) {
            c.status[inst] = st;
            c.active[inst] = 0;
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int ticket = atomicAdd(c.counter, 1u);
        last_block = ticket == (unsigned int)(c.n_inst - 1);
    }
    __syncthreads();
    if (!last_block || threadIdx.x != 0) return;
    __threadfence();
    int any = 0;
    for (int i = 0; i < c.n_inst; ++i) any |= __ldcg(c.active + i);
    *c.any_active = any;
    *c.counter = 0u;
    if (use_cond) cudaGraphSetConditional(h, any ? 1u : 0u);
}

}  // namespace

// ------------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------------
cudaError_t launch_force_b(const FomB& g, const int* active, int scatter, cudaStream_t s, const TraceFuse* trp) {
    if (g.n_eblk == 0) return cudaSuccess;
    const int b = g.eblock;
    TraceFuse tr;
    if (trp) tr = *trp;
    long long items = 0;
    for (int k = 0; k < tr.n; ++k) items += 3LL * tr.c[k].R;
    const int grid = g.n_eblk + (int)((items + b - 1) / b);
    if (g.df32) return launch_force_df_b(g, active, tr, s);
#define OSAM_LAUNCH(MAT, T, MODE) k_force_b<MAT, T, MODE><<<grid, b, 0, s>>>(g, active, tr)
    const bool fp32 = g.fp32 != 0;
    if (g.tiled && !fp32) {
        long long titems = 0;
        for (int k = 0; k < tr.n; ++k) titems += 3LL * tr.c[k].R;
        const int tgrid = g.n_tblk + (int)((titems + 127) / 128);
        if (g.occ && scatter == kGather) {
            if (g.material == OSAM_NEO_HOOKEAN) k_force_tile_occ_b<OSAM_NEO_HOOKEAN><<<tgrid, 128, 0, s>>>(g, active, tr);
            else if (g.material == OSAM_SAINT_VENANT_KIRCHHOFF)
                k_force_tile_occ_b<OSAM_SAINT_VENANT_KIRCHHOFF><<<tgrid, 128, 0, s>>>(g, active, tr);
            else k_force_tile_occ_b<OSAM_LINEAR_ELASTIC><<<tgrid, 128, 0, s>>>(g, active, tr);
            return cudaGetLastError();
        }
        if (g.material == OSAM_NEO_HOOKEAN) {
            if (scatter == kAtomic) k_force_tile_b<OSAM_NEO_HOOKEAN, kAtomic><<<tgrid, 128, 0, s>>>(g, active, tr);
            else k_force_tile_b<OSAM_NEO_HOOKEAN, kGather><<<tgrid, 128, 0, s>>>(g, active, tr);
        } else if (g.material == OSAM_SAINT_VENANT_KIRCHHOFF) {
            if (scatter == kAtomic) k_force_tile_b<OSAM_SAINT_VENANT_KIRCHHOFF, kAtomic><<<tgrid, 128, 0, s>>>(g, active, tr);
            else k_force_tile_b<OSAM_SAINT_VENANT_KIRCHHOFF, kGather><<<tgrid, 128, 0, s>>>(g, active, tr);
        } else {
            if (scatter == kAtomic) k_force_tile_b<OSAM_LINEAR_ELASTIC, kAtomic><<<tgrid, 128, 0, s>>>(g, active, tr);
            else k_force_tile_b<OSAM_LINEAR_ELASTIC, kGather><<<tgrid, 128, 0, s>>>(g, active, tr);
        }
        return cudaGetLastError();
    }
    if (g.occ && !fp32 && scatter == kGather && b <= 128) {
        if (g.material == OSAM_NEO_HOOKEAN) k_force_occ_b<OSAM_NEO_HOOKEAN><<<grid, b, 0, s>>>(g, active, tr);
        else if (g.material == OSAM_SAINT_VENANT_KIRCHHOFF) k_force_occ_b<OSAM_SAINT_VENANT_KIRCHHOFF><<<grid, b, 0, s>>>(g, active, tr);
        else k_force_occ_b<OSAM_LINEAR_ELASTIC><<<grid, b, 0, s>>>(g, active, tr);
        return cudaGetLastError();
    }
    if (g.material == OSAM_NEO_HOOKEAN) {
        if (fp32) { if (scatter == kAtomic) OSAM_LAUNCH(OSAM_NEO_HOOKEAN, float, kAtomic); else OSAM_LAUNCH(OSAM_NEO_HOOKEAN, float, kGather); }
        else { if (scatter == kAtomic) OSAM_LAUNCH(OSAM_NEO_HOOKEAN, double, kAtomic); else OSAM_LAUNCH(OSAM_NEO_HOOKEAN, double, kGather); }
    } else if (g.material == OSAM_SAINT_VENANT_KIRCHHOFF) {
        if (fp32) { if (scatter == kAtomic) OSAM_LAUNCH(OSAM_SAINT_VENANT_KIRCHHOFF, float, kAtomic); else OSAM_LAUNCH(OSAM_SAINT_VENANT_KIRCHHOFF, float, kGather); }
        else { if (scatter == kAtomic) OSAM_LAUNCH(OSAM_SAINT_VENANT_KIRCHHOFF, double, kAtomic); else OSAM_LAUNCH(OSAM_SAINT_VENANT_KIRCHHOFF, double, kGather); }
    } else {
        if (fp32) { if (scatter == kAtomic) OSAM_LAUNCH(OSAM_LINEAR_ELASTIC, float, kAtomic); else OSAM_LAUNCH(OSAM_LINEAR_ELASTIC, float, kGather); }
        else { if (scatter == kAtomic) OSAM_LAUNCH(OSAM_LINEAR_ELASTIC, double, kAtomic); else OSAM_LAUNCH(OSAM_LINEAR_ELASTIC, double, kGather); }
    }
#undef OSAM_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_force_init_b(const FomB& g, const int* active, cudaStream_t s) {
    if (g.n_eblk == 0) return cudaSuccess;
    k_scale_u0_b<<<g.n_nblk, kNodeBlock, 0, s>>>(g, active);
    if (g.material == OSAM_NEO_HOOKEAN)
        k_force_b<OSAM_NEO_HOOKEAN, double, kGather><<<g.n_eblk, g.eblock, 0, s>>>(g, active, TraceFuse{});
    else if (g.material == OSAM_SAINT_VENANT_KIRCHHOFF)
        k_force_b<OSAM_SAINT_VENANT_KIRCHHOFF, double, kGather><<<g.n_eblk, g.eblock, 0, s>>>(g, active, TraceFuse{});
    else
        k_force_b<OSAM_LINEAR_ELASTIC, double, kGather><<<g.n_eblk, g.eblock, 0, s>>>(g, active, TraceFuse{});
    return cudaGetLastError();
}

cudaError_t launch_init_accel_b(const FomB& g, const int* active, cudaStream_t s) {
    k_init_accel_b<<<g.n_nblk, kNodeBlock, 0, s>>>(g, active);
    return cudaGetLastError();
}

cudaError_t launch_node_b(const FomB& g, const int* active, int scatter, int slot1, int slot2, int predict_only,
                          const double* ucur, double* unext, double dt, cudaStream_t s) {
    const bool fp32 = g.fp32 != 0;
    if (g.df32) return launch_node_df_b(g, active, slot1, slot2, predict_only, ucur, unext, dt, s);
    if (fp32) {
        if (scatter == kAtomic) k_node_b<float, kAtomic><<<g.n_nblk, kNodeBlock, 0, s>>>(g, active, slot1, slot2, predict_only, ucur, unext, dt);
        else k_node_b<float, kGather><<<g.n_nblk, kNodeBlock, 0, s>>>(g, active, slot1, slot2, predict_only, ucur, unext, dt);
    } else {
        if (scatter == kAtomic) k_node_b<double, kAtomic><<<g.n_nblk, kNodeBlock, 0, s>>>(g, active, slot1, slot2, predict_only, ucur, unext, dt);
        else k_node_b<double, kGather><<<g.n_nblk, kNodeBlock, 0, s>>>(g, active, slot1, slot2, predict_only, ucur, unext, dt);
    }
    return cudaGetLastError();
}

cudaError_t launch_saverest_fom_b(const FomB& g, const int* active, int restore, cudaStream_t s) {
    k_saverest_fom_b<<<g.n_nblk, kNodeBlock, 0, s>>>(g, active, restore);
    return cudaGetLastError();
}

cudaError_t launch_copy_u10_b(const FomB& g, const int* active, cudaStream_t s) {
    k_copy_u10_b<<<g.n_nblk, kNodeBlock, 0, s>>>(g, active);
    return cudaGetLastError();
}

cudaError_t launch_norms_fom_b(const FomB& g, const int* active, double dt, cudaStream_t s) {
    k_norms_fom_b<<<g.n_nblk, kNodeBlock, 0, s>>>(g, active, dt);
    return cudaGetLastError();
}

cudaError_t launch_trace_b(const CplB& c, const int* active, const FomB& src, const double* u, int slot,
                           cudaStream_t s) {
    if (c.R == 0) return cudaSuccess;
    k_trace_b<<<grid_for(3LL * c.R, 128), 128, 0, s>>>(c, active, src, u, slot);
    return cudaGetLastError();
}

cudaError_t launch_publish_b(const CplB& c, const int* active, int slot0, int nslots, int ns, int nd, cudaStream_t s) {
    if (c.R == 0 || nslots <= 0) return cudaSuccess;
    if (ns < 1 || nd < 1 || slot0 < 0 || slot0 + nslots > nd + 1) return cudaErrorInvalidValue;
    k_publish_b<<<grid_for(9LL * c.R * nslots, 256), 256, 0, s>>>(c, active, slot0, nslots, ns, nd);
    return cudaGetLastError();
}

cudaError_t launch_zoh_fom_b(const CplB& c, const int* active, const FomB& src, int nsub, cudaStream_t s) {
    if (c.R == 0) return cudaSuccess;
    k_zoh_fom_b<<<grid_for(3LL * c.R, 128), 128, 0, s>>>(c, active, src, nsub + 1);
    return cudaGetLastError();
}

cudaError_t launch_rom_record0_b(const RomB& r, const int* active, cudaStream_t s) {
    k_rom_record0_b<<<r.n_inst, 128, 0, s>>>(r, active);
    return cudaGetLastError();
}

cudaError_t launch_rom_project_b(const RomB& r, const int* active, int slot0, int slot1, cudaStream_t s) {
    if (r.rs_max == 0 || slot1 < slot0) return cudaSuccess;
    dim3 g(r.rs_max, slot1 - slot0 + 1, r.n_inst);
    k_rom_project_b<<<g, 128, 0, s>>>(r, active, slot0);
    return cudaGetLastError();
}

cudaError_t launch_rom_step_b(const RomB& r, const int* active, int slot, double dt, int rhs_only, cudaStream_t s) {
    if (r.r_max > kMaxR) return cudaErrorInvalidValue;
    dim3 g(r.gx_max, r.gy_max, r.n_inst);
    k_rom_step_b<<<g, kRomBlock, 0, s>>>(r, active, slot, dt, rhs_only);
    return cudaGetLastError();
}

cudaError_t launch_rom_reconstruct_b(const CplB& c, const int* active, const RomB& src, int zoh, int ns, int nd,
                                     cudaStream_t s) {
    if (c.R == 0) return cudaSuccess;
    if (ns < 1 || nd < 1) return cudaErrorInvalidValue;
    if (zoh) {
        dim3 g(grid_for(3LL * c.R, 128), nd + 1, 3);
        k_rom_reconstruct_b<<<g, 128, 0, s>>>(c, active, src, 1, 0, ns, nd);
    } else {
        dim3 g(grid_for(3LL * c.R, 128), nd, 3);
        k_rom_reconstruct_b<<<g, 128, 0, s>>>(c, active, src, 0, 1, ns, nd);
    }
    return cudaGetLastError();
}

cudaError_t launch_rom_norms_b(const RomB& r, const int* active, double dt, cudaStream_t s) {
    k_rom_norms_b<<<r.n_inst, 128, 0, s>>>(r, active, dt);
    return cudaGetLastError();
}

cudaError_t launch_saverest_rom_b(const RomB& r, const int* active, int restore, cudaStream_t s) {
    k_saverest_rom_b<<<r.n_inst, 128, 0, s>>>(r, active, restore);
    return cudaGetLastError();
}

cudaError_t launch_reset_ctl(const CtlB& c, cudaStream_t s) {
    k_reset_ctl<<<grid_for(c.n_inst, 128), 128, 0, s>>>(c);
    return cudaGetLastError();
}

cudaError_t launch_controller(const CtlB& c, cudaGraphConditionalHandle h, int use_cond, cudaStream_t s) {
    k_controller<<<c.n_inst, 256, 0, s>>>(c, h, use_cond);
    return cudaGetLastError();
}

}  // namespace osam
