// Tangent action of the implicit Newton systems: K(u) p, the directional derivative of the hex8
// internal force at u along p (Appendix A tangents: A.1 linear elastic, A.2 Saint Venant-Kirchhoff,
// A.3 Neo-Hookean through the directional derivative of P in cofactor form), in the sum
// factorisation of the force kernels:
// edge differences and two-stage interpolation of u and p to the 2x2x2 Gauss points, dP there, the
// transposed interpolation back to the 8 nodes.  Output in the element-buffer layout [24][NE] of the
// gather scheme, so the node kernels sum it in a fixed order.
#include <cuda_runtime.h>

#include "hex8_math.cuh"
#include "nh_tangent.cuh"
#include "osam_internal.h"

namespace osam {

namespace {

using namespace hex8;

__device__ __forceinline__ bool run_inst(const int* mask, int inst) { return !mask || mask[inst]; }

// Saint Venant-Kirchhoff (A.2): dP = G S + F dS, dS = lam tr(dE) I + 2 mu dE, dE = sym(F^T G)
// (lam, mu pre-scaled; F = I + H)
__device__ __forceinline__ void svk_tangent(const double H[3][3], const double G[3][3], double lam, double mu,
                                            double dP[3][3]) {
    double S[3][3], dS[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            double e = H[i][j] + H[j][i], de = G[i][j] + G[j][i];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                e = fma(H[k][i], H[k][j], e);
                de = fma(H[k][i], G[k][j], fma(G[k][i], H[k][j], de));
            }
            S[i][j] = 0.5 * e;
            dS[i][j] = 0.5 * de;
        }
    const double lt = lam * (S[0][0] + S[1][1] + S[2][2]), dlt = lam * (dS[0][0] + dS[1][1] + dS[2][2]);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            S[i][j] = i == j ? fma(2.0 * mu, S[i][j], lt) : 2.0 * mu * S[i][j];
            dS[i][j] = i == j ? fma(2.0 * mu, dS[i][j], dlt) : 2.0 * mu * dS[i][j];
            if (j != i) { S[j][i] = S[i][j]; dS[j][i] = dS[i][j]; }
        }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double p = dS[i][j];
#pragma unroll
            for (int k = 0; k < 3; ++k) p = fma(G[i][k], S[k][j], fma(H[i][k], dS[k][j], p));
            dP[i][j] = p;
        }
}

// element tangent action: the directional derivative of the element forces at u along p, written
// to the element buffer (same layout and sum factorisation as the force kernels)
template <int MAT>
__global__ void __launch_bounds__(256) k_tangent_b(const FomB g, const int* __restrict__ mask) {
    const int2 b = g.eblk[blockIdx.x];
    if (!run_inst(mask, b.x)) return;
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
    double Dx[3][2][2], Dy[3][2][2], Dz[3][2][2], Ex[3][2][2], Ey[3][2][2], Ez[3][2][2];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double U[8], P[8];
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8) {
            const long long d = (long long)c * g.NN + I.node_off + node[c8];
            U[c8] = g.us[d];
            P[c8] = g.cg_p[d] * I.invh;
        }
        edge_differences_prescaled<double>(U, Dx[c], Dy[c], Dz[c]);
        edge_differences_prescaled<double>(P, Ex[c], Ey[c], Ez[c]);
    }
    double Gx[3][2][2], Gy[3][2][2], Gz[3][2][2], Bx[3][2][2], By[3][2][2], Bz[3][2][2];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        lerp2<double>(Dx[c], Gx[c]); lerp2<double>(Dy[c], Gy[c]); lerp2<double>(Dz[c], Gz[c]);
        lerp2<double>(Ex[c], Bx[c]); lerp2<double>(Ey[c], By[c]); lerp2<double>(Ez[c], Bz[c]);
    }
    const double lam = I.lam_e ? I.lam_e[e] : I.lam;
    const double mu = I.mu_e ? I.mu_e[e] : I.mu;
    double m1, m2, m3;
    if (MAT == OSAM_NEO_HOOKEAN) {
        const double kappa = lam + (2.0 / 3.0) * mu;
        m1 = 0.5 * kappa * I.w8; m2 = mu * I.w8; m3 = mu * I.w8 / 3.0;
    } else {
        m1 = lam * I.w8; m2 = mu * I.w8; m3 = 0.0;
    }
    double Sx[3][2][2], Sy[3][2][2], Sz[3][2][2];
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                double Hm[3][3], Gm[3][3], dP[3][3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    Hm[c][0] = Gx[c][q][r]; Hm[c][1] = Gy[c][p][r]; Hm[c][2] = Gz[c][p][q];
                    Gm[c][0] = Bx[c][q][r]; Gm[c][1] = By[c][p][r]; Gm[c][2] = Bz[c][p][q];
                }
                if (MAT == OSAM_NEO_HOOKEAN) {
                    double pk, pm;
                    tangent::nh_tangent(Hm, Gm, m1, m2, m3, dP, pk, pm);
                } else if (MAT == OSAM_SAINT_VENANT_KIRCHHOFF) {
                    svk_tangent(Hm, Gm, m1, m2, dP);
                } else {
                    stress_le<double>(Gm, m1, m2, dP);  // linear: the tangent applied to G is sigma(G)
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (p == 0) Sx[c][q][r] = dP[c][0]; else Sx[c][q][r] += dP[c][0];
                    if (q == 0) Sy[c][p][r] = dP[c][1]; else Sy[c][p][r] += dP[c][1];
                    if (r == 0) Sz[c][p][q] = dP[c][2]; else Sz[c][p][q] += dP[c][2];
                }
            }
    double* fe = static_cast<double*>(g.fe) + I.elem_off;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double Fc[8], Tm[2][2];
        lerp2T<double>(Sx[c], Tm);
#pragma unroll
        for (int ay = 0; ay < 2; ++ay)
#pragma unroll
            for (int az = 0; az < 2; ++az) { Fc[1 + 2 * ay + 4 * az] = Tm[ay][az]; Fc[2 * ay + 4 * az] = -Tm[ay][az]; }
        lerp2T<double>(Sy[c], Tm);
#pragma unroll
        for (int ax = 0; ax < 2; ++ax)
#pragma unroll
            for (int az = 0; az < 2; ++az) { Fc[ax + 2 + 4 * az] += Tm[ax][az]; Fc[ax + 4 * az] -= Tm[ax][az]; }
        lerp2T<double>(Sz[c], Tm);
#pragma unroll
        for (int ax = 0; ax < 2; ++ax)
#pragma unroll
            for (int ay = 0; ay < 2; ++ay) { Fc[ax + 2 * ay + 4] += Tm[ax][ay]; Fc[ax + 2 * ay] -= Tm[ax][ay]; }
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8) fe[(long long)(c8 * 3 + c) * g.NE + e] = Fc[c8];
    }
}

// ---- Neo-Hookean Newton linearisation stored once per Newton step --------------------------------
// The tangent at u is applied ~6 times per Newton step (CG iterations) while u stays fixed, so the
// u-dependent part of dP = dbeta cof + beta dcof[G] + dalpha F + alpha G is computed once, with the
// force of the Newton residual, and stored per Gauss point: F, cof F, alpha, beta and the two
// coefficients of the scalar derivatives, dalpha = a1 dJ and dbeta = b1 dJ + a1 (F : G), dJ = cof : G,
//   a1 = -2/3 alpha / J,  b1 = 2 kappa/2 - (a1 trC / 3 + beta) / J   (from P = alpha F + beta cof,
//   alpha = mu J^-2/3, beta = (kappa/2 (J^2 - 1) - mu/3 J^-2/3 trC) / J).
// Layout [kLinPerGp][8 Gauss points][NE], element index fastest (coalesced): F (9), cof F (9), alpha,
// beta, a1, b1.
static_assert(kLinPerGp == 22, "stored linearisation: F, cof F, alpha, beta, a1, b1");

__device__ __forceinline__ void nodal_grads(const FomB& g, const InstFom& I, const double* x, double scale,
                                            const int node[8], double Gx[3][2][2], double Gy[3][2][2],
                                            double Gz[3][2][2]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double V[8], Dx[2][2], Dy[2][2], Dz[2][2];
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8) V[c8] = x[(long long)c * g.NN + I.node_off + node[c8]] * scale;
        edge_differences_prescaled<double>(V, Dx, Dy, Dz);
        lerp2<double>(Dx, Gx[c]); lerp2<double>(Dy, Gy[c]); lerp2<double>(Dz, Gz[c]);
    }
}

// transposed interpolation of the Gauss-point sums (scaled like the force's: Walsh basis, factor 4 in
// the material factors) and the element-buffer write
template <typename T>
__device__ __forceinline__ void write_element(T* fe, long long ne, int e, const T Sx[3][2][2], const T Sy[3][2][2],
                                              const T Sz[3][2][2]) {
    T F[3][8];
    walsh_transpose<T>(Sx, Sy, Sz, F);
#pragma unroll
    for (int c8 = 0; c8 < 8; ++c8)
#pragma unroll
        for (int c = 0; c < 3; ++c) fe[(long long)(c8 * 3 + c) * ne + e] = F[c][c8];
}

struct ElemIdx {
    InstFom I;
    int e;
    int node[8];
    bool ok;
};

__device__ __forceinline__ ElemIdx elem_idx(const FomB& g, const int* mask) {
    ElemIdx x;
    const int2 b = g.eblk[blockIdx.x];
    x.ok = run_inst(mask, b.x);
    x.I = g.inst[b.x];
    x.e = b.y + threadIdx.x;
    x.ok = x.ok && x.e < x.I.ne;
    if (!x.ok) return x;
    const int i = x.e % x.I.nx;
    const int t = x.e / x.I.nx;
    const int j = t % x.I.ny;
    const int k = t / x.I.ny;
    const int sy = x.I.nx + 1, sz = (x.I.nx + 1) * (x.I.ny + 1);
    const int n0 = i + sy * j + sz * k;
#pragma unroll
    for (int c8 = 0; c8 < 8; ++c8) x.node[c8] = n0 + (c8 & 1) + ((c8 >> 1) & 1) * sy + ((c8 >> 2) & 1) * sz;
    return x;
}

// FP64 -> FP32 for the stored FP32 linearisation by integer operations (f32_rz: a conversion
// instruction would take a slot of the FP64 pipe, the bound of the Newton force, 176 times per
// element; the entries -- F, cof F and the material-scaled factors -- lie far inside the FP32 range,
// and the rounding toward zero is at the CG operator's own FP32 level).
__device__ __forceinline__ double lin_value(double x, double*) { return x; }
__device__ __forceinline__ float lin_value(double x, float*) { return f32_rz(x); }

// The per-Gauss-point quantities of the Newton linearisation, stored by the Neo-Hookean Gauss sums'
// hook (TL: the storage type); a1 and b1 from the force's own 1/J (the cube of its reciprocal cube
// root, no division).  Material factors scaled by h^2/32 like the force's (the Walsh-basis transposed
// interpolation carries the remaining factor 4), so the tangent's dP is scaled alike.
template <typename TL>
struct LinStore {
    TL* lin;             // this element's first entry
    long long st;        // stride between quantities (8 NE)
    long long ne;        // stride between Gauss points (NE)
    double kap2;         // m1 of the material factors
    __device__ __forceinline__ void operator()(int p, int q, int r, const double (&Fm)[3][3], const double (&Cm)[3][3],
                                               double J, double trC, double invJ, double alpha, double beta) const {
        (void)J;
        const double a1 = -(2.0 / 3.0) * alpha * invJ;
        const double b1 = 2.0 * kap2 - invJ * fma(a1, trC * (1.0 / 3.0), beta);
        TL* lg = lin + (long long)(4 * p + 2 * q + r) * ne;
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            lg[a * st] = lin_value(Fm[a / 3][a % 3], lg);
            lg[(9 + a) * st] = lin_value(Cm[a / 3][a % 3], lg);
        }
        lg[18 * st] = lin_value(alpha, lg); lg[19 * st] = lin_value(beta, lg);
        lg[20 * st] = lin_value(a1, lg); lg[21 * st] = lin_value(b1, lg);
    }
};

// Newton residual force of a Neo-Hookean group at u (from u / h) plus the stored linearisation: the
// explicit force's arithmetic (1 of F's diagonal in the first interpolation stage, paired Gauss-point
// sums, Walsh-basis transposed interpolation) with the linearisation written at each Gauss point
template <typename TL>
__global__ void __launch_bounds__(256) k_force_lin_b(const FomB g, TL* __restrict__ lin_base,
                                                     const int* __restrict__ mask) {
    const ElemIdx x = elem_idx(g, mask);
    if (!x.ok) return;
    const InstFom& I = x.I;
    const int e = x.e;
    double Gx[3][2][2], Gy[3][2][2], Gz[3][2][2];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double V[8], Dx[2][2], Dy[2][2], Dz[2][2];
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8) V[c8] = g.us[(long long)c * g.NN + I.node_off + x.node[c8]];
        edge_differences_prescaled<double>(V, Dx, Dy, Dz);
        lerp2<double>(Dx, Gx[c], c == 0);
        lerp2<double>(Dy, Gy[c], c == 1);
        lerp2<double>(Dz, Gz[c], c == 2);
    }
    double m1, m2, m3;
    if (I.lam_e || I.mu_e)
        material_factors<OSAM_NEO_HOOKEAN, double>(I.lam_e ? I.lam_e[e] : I.lam, I.mu_e ? I.mu_e[e] : I.mu, I.wq,
                                                   I.wq3, m1, m2, m3);
    else { m1 = I.m1; m2 = I.m2; m3 = I.m3; }
    const LinStore<TL> store{lin_base + I.elem_off + e, 8LL * g.NE, g.NE, m1};
    double Sx[3][2][2], Sy[3][2][2], Sz[3][2][2], F[3][8];
    nh_gauss_sums<double>(Gx, Gy, Gz, m1, m2, m3, Sx, Sy, Sz, store);
    walsh_transpose<double>(Sx, Sy, Sz, F);
    double* fe = static_cast<double*>(g.fe) + I.elem_off;
#pragma unroll
    for (int c8 = 0; c8 < 8; ++c8)
#pragma unroll
        for (int c = 0; c < 3; ++c) fe[(long long)(c8 * 3 + c) * g.NE + e] = F[c][c8];
}

// tangent action from the stored linearisation: per Gauss point 166 FP64 flops instead of 243, and
// no interpolation of u
__global__ void __launch_bounds__(256) k_tangent_lin_b(const FomB g, const int* __restrict__ mask) {
    const ElemIdx x = elem_idx(g, mask);
    if (!x.ok) return;
    const InstFom& I = x.I;
    const int e = x.e;
    double Bx[3][2][2], By[3][2][2], Bz[3][2][2];
    nodal_grads(g, I, g.cg_p, I.invh, x.node, Bx, By, Bz);
    const double* lin = g.lin + I.elem_off + e;
    const long long st = 8LL * g.NE;
    double Sx[3][2][2], Sy[3][2][2], Sz[3][2][2];
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int gp = 4 * p + 2 * q + r;
                const double* lg = lin + (long long)gp * g.NE;
                double F[3][3], cf[3][3], G[3][3], dc[3][3];
#pragma unroll
                for (int a = 0; a < 9; ++a) {
                    F[a / 3][a % 3] = __ldg(lg + a * st);
                    cf[a / 3][a % 3] = __ldg(lg + (9 + a) * st);
                }
                const double alpha = __ldg(lg + 18 * st), beta = __ldg(lg + 19 * st);
                const double a1 = __ldg(lg + 20 * st), b1 = __ldg(lg + 21 * st);
#pragma unroll
                for (int c = 0; c < 3; ++c) { G[c][0] = Bx[c][q][r]; G[c][1] = By[c][p][r]; G[c][2] = Bz[c][p][q]; }
                double dJ = 0.0, FG = 0.0;
#pragma unroll
                for (int a = 0; a < 9; ++a) {
                    dJ = fma(cf[a / 3][a % 3], G[a / 3][a % 3], dJ);
                    FG = fma(F[a / 3][a % 3], G[a / 3][a % 3], FG);
                }
                dc[0][0] = G[1][1] * F[2][2] + F[1][1] * G[2][2] - G[1][2] * F[2][1] - F[1][2] * G[2][1];
                dc[0][1] = G[1][2] * F[2][0] + F[1][2] * G[2][0] - G[1][0] * F[2][2] - F[1][0] * G[2][2];
                dc[0][2] = G[1][0] * F[2][1] + F[1][0] * G[2][1] - G[1][1] * F[2][0] - F[1][1] * G[2][0];
                dc[1][0] = G[0][2] * F[2][1] + F[0][2] * G[2][1] - G[0][1] * F[2][2] - F[0][1] * G[2][2];
                dc[1][1] = G[0][0] * F[2][2] + F[0][0] * G[2][2] - G[0][2] * F[2][0] - F[0][2] * G[2][0];
                dc[1][2] = G[0][1] * F[2][0] + F[0][1] * G[2][0] - G[0][0] * F[2][1] - F[0][0] * G[2][1];
                dc[2][0] = G[0][1] * F[1][2] + F[0][1] * G[1][2] - G[0][2] * F[1][1] - F[0][2] * G[1][1];
                dc[2][1] = G[0][2] * F[1][0] + F[0][2] * G[1][0] - G[0][0] * F[1][2] - F[0][0] * G[1][2];
                dc[2][2] = G[0][0] * F[1][1] + F[0][0] * G[1][1] - G[0][1] * F[1][0] - F[0][1] * G[1][0];
                const double dalpha = a1 * dJ;
                const double dbeta = fma(b1, dJ, a1 * FG);
                double dP[3][3];
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b2 = 0; b2 < 3; ++b2)
                        dP[a][b2] = fma(dbeta, cf[a][b2], fma(beta, dc[a][b2], fma(dalpha, F[a][b2], alpha * G[a][b2])));
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (p == 0) Sx[c][q][r] = dP[c][0]; else Sx[c][q][r] += dP[c][0];
                    if (q == 0) Sy[c][p][r] = dP[c][1]; else Sy[c][p][r] += dP[c][1];
                    if (r == 0) Sz[c][p][q] = dP[c][2]; else Sz[c][p][q] += dP[c][2];
                }
            }
    write_element<double>(static_cast<double*>(g.fe) + I.elem_off, g.NE, e, Sx, Sy, Sz);
}

// The tangent action of k_tangent_lin_b in FP32 (OSAM_FP64_TANGENT32): the linearisation read as
// stored in FP32 (half the bytes), the direction p converted once per nodal value, every Gauss-point
// operation on the FP32 pipes, and the element contributions written in FP32 to the FP32 element
// buffer (the CG's Ap kernel sums them in FP32 and adds them to its FP64 mass term).  p is converted
// with the integer-only f32_rz, so no FP64-pipe instruction is left.
__global__ void __launch_bounds__(256) k_tangent_lin32_b(const FomB g, const int* __restrict__ mask) {
    const ElemIdx x = elem_idx(g, mask);
    if (!x.ok) return;
    const InstFom& I = x.I;
    const int e = x.e;
    const float sc = float(I.invh);
    float Bx[3][2][2], By[3][2][2], Bz[3][2][2];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float V[8], Dx[2][2], Dy[2][2], Dz[2][2];
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8)
            V[c8] = f32_rz(g.cg_p[(long long)c * g.NN + I.node_off + x.node[c8]]) * sc;
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                Dx[a][b] = V[1 + 2 * a + 4 * b] - V[2 * a + 4 * b];
                Dy[a][b] = V[a + 2 + 4 * b] - V[a + 4 * b];
                Dz[a][b] = V[a + 2 * b + 4] - V[a + 2 * b];
            }
        lerp2<float>(Dx, Bx[c]); lerp2<float>(Dy, By[c]); lerp2<float>(Dz, Bz[c]);
    }
    const float* lin = g.linf + I.elem_off + e;
    const long long st = 8LL * g.NE;
    float Sx[3][2][2], Sy[3][2][2], Sz[3][2][2];
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int gp = 4 * p + 2 * q + r;
                const float* lg = lin + (long long)gp * g.NE;
                float F[3][3], cf[3][3], G[3][3], dc[3][3];
#pragma unroll
                for (int a = 0; a < 9; ++a) {
                    F[a / 3][a % 3] = __ldg(lg + a * st);
                    cf[a / 3][a % 3] = __ldg(lg + (9 + a) * st);
                }
                const float alpha = __ldg(lg + 18 * st), beta = __ldg(lg + 19 * st);
                const float a1 = __ldg(lg + 20 * st), b1 = __ldg(lg + 21 * st);
#pragma unroll
                for (int c = 0; c < 3; ++c) { G[c][0] = Bx[c][q][r]; G[c][1] = By[c][p][r]; G[c][2] = Bz[c][p][q]; }
                float dJ = 0.f, FG = 0.f;
#pragma unroll
                for (int a = 0; a < 9; ++a) {
                    dJ = fmaf(cf[a / 3][a % 3], G[a / 3][a % 3], dJ);
                    FG = fmaf(F[a / 3][a % 3], G[a / 3][a % 3], FG);
                }
                dc[0][0] = G[1][1] * F[2][2] + F[1][1] * G[2][2] - G[1][2] * F[2][1] - F[1][2] * G[2][1];
                dc[0][1] = G[1][2] * F[2][0] + F[1][2] * G[2][0] - G[1][0] * F[2][2] - F[1][0] * G[2][2];
                dc[0][2] = G[1][0] * F[2][1] + F[1][0] * G[2][1] - G[1][1] * F[2][0] - F[1][1] * G[2][0];
                dc[1][0] = G[0][2] * F[2][1] + F[0][2] * G[2][1] - G[0][1] * F[2][2] - F[0][1] * G[2][2];
                dc[1][1] = G[0][0] * F[2][2] + F[0][0] * G[2][2] - G[0][2] * F[2][0] - F[0][2] * G[2][0];
                dc[1][2] = G[0][1] * F[2][0] + F[0][1] * G[2][0] - G[0][0] * F[2][1] - F[0][0] * G[2][1];
                dc[2][0] = G[0][1] * F[1][2] + F[0][1] * G[1][2] - G[0][2] * F[1][1] - F[0][2] * G[1][1];
                dc[2][1] = G[0][2] * F[1][0] + F[0][2] * G[1][0] - G[0][0] * F[1][2] - F[0][0] * G[1][2];
                dc[2][2] = G[0][0] * F[1][1] + F[0][0] * G[1][1] - G[0][1] * F[1][0] - F[0][1] * G[1][0];
                const float dalpha = a1 * dJ;
                const float dbeta = fmaf(b1, dJ, a1 * FG);
                float dP[3][3];
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b2 = 0; b2 < 3; ++b2)
                        dP[a][b2] = fmaf(dbeta, cf[a][b2], fmaf(beta, dc[a][b2], fmaf(dalpha, F[a][b2], alpha * G[a][b2])));
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (p == 0) Sx[c][q][r] = dP[c][0]; else Sx[c][q][r] += dP[c][0];
                    if (q == 0) Sy[c][p][r] = dP[c][1]; else Sy[c][p][r] += dP[c][1];
                    if (r == 0) Sz[c][p][q] = dP[c][2]; else Sz[c][p][q] += dP[c][2];
                }
            }
    write_element<float>(g.fe32 + I.elem_off, g.NE, e, Sx, Sy, Sz);
}

}  // namespace

cudaError_t launch_force_lin_b(const FomB& g, const int* mask, cudaStream_t s) {
    if (g.n_eblk == 0) return cudaSuccess;
    if (g.eblock > 256 || (!g.lin && !g.linf) || g.material != OSAM_NEO_HOOKEAN) return cudaErrorInvalidValue;
    if (g.linf) k_force_lin_b<float><<<g.n_eblk, g.eblock, 0, s>>>(g, g.linf, mask);
    else k_force_lin_b<double><<<g.n_eblk, g.eblock, 0, s>>>(g, g.lin, mask);
    return cudaGetLastError();
}

cudaError_t launch_tangent_lin_b(const FomB& g, const int* mask, cudaStream_t s) {
    if (g.n_eblk == 0) return cudaSuccess;
    if (g.eblock > 256 || g.material != OSAM_NEO_HOOKEAN) return cudaErrorInvalidValue;
    if (g.linf && g.fe32) k_tangent_lin32_b<<<g.n_eblk, g.eblock, 0, s>>>(g, mask);
    else if (g.lin) k_tangent_lin_b<<<g.n_eblk, g.eblock, 0, s>>>(g, mask);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_tangent_b(const FomB& g, const int* mask, cudaStream_t s) {
    if (g.n_eblk == 0) return cudaSuccess;
    if (g.eblock > 256) return cudaErrorInvalidConfiguration;
    if (g.material == OSAM_NEO_HOOKEAN) k_tangent_b<OSAM_NEO_HOOKEAN><<<g.n_eblk, g.eblock, 0, s>>>(g, mask);
    else if (g.material == OSAM_SAINT_VENANT_KIRCHHOFF)
        k_tangent_b<OSAM_SAINT_VENANT_KIRCHHOFF><<<g.n_eblk, g.eblock, 0, s>>>(g, mask);
    else k_tangent_b<OSAM_LINEAR_ELASTIC><<<g.n_eblk, g.eblock, 0, s>>>(g, mask);
    return cudaGetLastError();
}
}  // namespace osam
