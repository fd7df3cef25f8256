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

}  // namespace

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
