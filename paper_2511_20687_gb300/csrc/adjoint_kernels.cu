// Vector-Jacobian product of the hex8 internal force and the elementwise parts of the reverse
// sweep through the explicit central-difference rollout.
//
// For a hyperelastic law the tangent dP/dF has major symmetry, so the VJP of f with cotangent ybar
// at element level is the force-like contraction of the directional derivative dP[Gbar] with
// Gbar = grad(ybar):  ubar_b = sum_gp w detJ dP[Gbar] grad N_b.  Parameter cotangents are
// lambda_bar_e = sum_gp w detJ P_lambda : Gbar and mu_bar_e = sum_gp w detJ P_mu : Gbar.
// Neo-Hookean (cofactor form P = beta cof(F) + alpha F, alpha = mu J^-2/3,
// beta = [kappa/2 (J^2-1) - mu/3 J^-2/3 tr C] / J):
//   dJ = cof(F) : G,  d trC = 2 F : G,  d alpha = -2/3 alpha dJ / J,
//   d beta = [kappa J dJ - 1/3 (d alpha trC + alpha d trC)] / J - beta dJ / J,
//   dP = d beta cof + beta dcof[G] + d alpha F + alpha G,  dcof linear in G (cof is quadratic in F).
#include <cuda_runtime.h>

#include <cstdint>

#include "hex8_math.cuh"
#include "nh_tangent.cuh"
#include "osam_internal.h"

namespace osam {

namespace {

// scaled edge differences of a nodal field (see the forward kernel)
__device__ __forceinline__ void edge_diffs(const double* x, int sn, long long sc, const int node[8], double invh,
                                           double Dx[3][2][2], double Dy[3][2][2], double Dz[3][2][2]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double U[8];
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8) U[c8] = x[(long long)c * sc + (long long)node[c8] * sn] * invh;
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                Dx[c][p][q] = U[1 + 2 * p + 4 * q] - U[2 * p + 4 * q];
                Dy[c][p][q] = U[p + 2 + 4 * q] - U[p + 4 * q];
                Dz[c][p][q] = U[p + 2 * q + 4] - U[p + 2 * q];
            }
    }
}

using tangent::nh_tangent;

// One thread per element.  MODE kAtomic adds ubar into a.f ([3] x strided nodes); kGather writes the
// element's 24 contributions to the element buffer a.fe [24][ne] (corner-major, component), which a
// fixed-order gather sums per node (deterministic).  The transposed interpolation is the force's
// Walsh-basis stage (hex8::walsh_transpose), so the material factors carry its 1/4.
template <int MAT, int MODE>
__global__ void __launch_bounds__(128) k_hex8_vjp(const ElemArgs a, const double* ybar, int ysn, long long ysc,
                                                  double* lam_bar, double* mu_bar, int accumulate) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.ne) return;
    const int i = e % a.nx;
    const int t = e / a.nx;
    const int j = t % a.ny;
    const int k = t / a.ny;
    const int sy = a.nx + 1, sz = (a.nx + 1) * (a.ny + 1);
    const int n0 = i + sy * j + sz * k;
    int node[8];
#pragma unroll
    for (int c8 = 0; c8 < 8; ++c8) node[c8] = n0 + (c8 & 1) + ((c8 >> 1) & 1) * sy + ((c8 >> 2) & 1) * sz;
    const double lam = a.lam_e ? a.lam_e[e] : a.lam;
    const double mu = a.mu_e ? a.mu_e[e] : a.mu;
    double Dx[3][2][2], Dy[3][2][2], Dz[3][2][2];
    double Ex[3][2][2], Ey[3][2][2], Ez[3][2][2];
    edge_diffs(a.u, a.usn, a.usc, node, a.invh, Dx, Dy, Dz);
    edge_diffs(ybar, ysn, ysc, node, a.invh, Ex, Ey, Ez);
    double Gx[3][2][2], Gy[3][2][2], Gz[3][2][2], Bx[3][2][2], By[3][2][2], Bz[3][2][2];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        hex8::lerp2(Dx[c], Gx[c]); hex8::lerp2(Dy[c], Gy[c]); hex8::lerp2(Dz[c], Gz[c]);
        hex8::lerp2(Ex[c], Bx[c]); hex8::lerp2(Ey[c], By[c]); hex8::lerp2(Ez[c], Bz[c]);
    }
    double m1, m2, m3;
    hex8::material_factors<MAT, double>(lam, mu, a.wq, a.wq3, m1, m2, m3);
    double Sx[3][2][2], Sy[3][2][2], Sz[3][2][2];
    double lb = 0.0, mb = 0.0;
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
                    nh_tangent(Hm, Gm, m1, m2, m3, dP, pk, pm);
                    lb += pk;
                    mb = fma(2.0 / 3.0, pk, mb + pm);
                } else {
                    const double trG = Gm[0][0] + Gm[1][1] + Gm[2][2];
                    const double trH = Hm[0][0] + Hm[1][1] + Hm[2][2];
                    double symHG = 0.0;
#pragma unroll
                    for (int x = 0; x < 3; ++x)
#pragma unroll
                        for (int y = 0; y < 3; ++y) {
                            dP[x][y] = m2 * (Gm[x][y] + Gm[y][x]) + (x == y ? m1 * trG : 0.0);
                            symHG = fma(Hm[x][y] + Hm[y][x], Gm[x][y], symHG);
                        }
                    lb = fma(trH, trG, lb);
                    mb += symHG;
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (p == 0) Sx[c][q][r] = dP[c][0]; else Sx[c][q][r] += dP[c][0];
                    if (q == 0) Sy[c][p][r] = dP[c][1]; else Sy[c][p][r] += dP[c][1];
                    if (r == 0) Sz[c][p][q] = dP[c][2]; else Sz[c][p][q] += dP[c][2];
                }
            }
    double Fe[3][8];
    hex8::walsh_transpose<double>(Sx, Sy, Sz, Fe);
    if (MODE == kAtomic) {
        double* ub = static_cast<double*>(a.f);
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int c8 = 0; c8 < 8; ++c8) atomicAdd(ub + (long long)c * a.fsc + (long long)node[c8] * a.fsn, Fe[c][c8]);
    } else {
        double* fe = static_cast<double*>(a.fe);
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8)
#pragma unroll
            for (int c = 0; c < 3; ++c) fe[(long long)(c8 * 3 + c) * a.ne + e] = Fe[c][c8];
    }
    // w detJ = h^3/8 per Gauss point; Gbar above is the physical gradient
    const double vol8 = a.w8 / a.invh;
    if (lam_bar) lam_bar[e] = (accumulate ? lam_bar[e] : 0.0) + vol8 * lb;
    if (mu_bar) mu_bar[e] = (accumulate ? mu_bar[e] : 0.0) + vol8 * mb;
}

}  // namespace

cudaError_t launch_hex8_vjp(int material, int scatter, const ElemArgs& a, const double* ybar, int ysn, long long ysc,
                            double* lam_bar, double* mu_bar, int acc, cudaStream_t s) {
    if (a.ne <= 0) return cudaSuccess;
    const int g = grid_for(a.ne, 128);
    const bool at = scatter == kAtomic;
    if (material == OSAM_NEO_HOOKEAN) {
        if (at) k_hex8_vjp<OSAM_NEO_HOOKEAN, kAtomic><<<g, 128, 0, s>>>(a, ybar, ysn, ysc, lam_bar, mu_bar, acc);
        else k_hex8_vjp<OSAM_NEO_HOOKEAN, kGather><<<g, 128, 0, s>>>(a, ybar, ysn, ysc, lam_bar, mu_bar, acc);
    } else {
        if (at) k_hex8_vjp<OSAM_LINEAR_ELASTIC, kAtomic><<<g, 128, 0, s>>>(a, ybar, ysn, ysc, lam_bar, mu_bar, acc);
        else k_hex8_vjp<OSAM_LINEAR_ELASTIC, kGather><<<g, 128, 0, s>>>(a, ybar, ysn, ysc, lam_bar, mu_bar, acc);
    }
    return cudaGetLastError();
}

}  // namespace osam

namespace osam {
namespace {

// reverse of the corrector v' = v + dt/2 (a + a'), a' = -M^-1 f(u'):  abar' += dt/2 vbar;
// y = -M^-1 abar' (free dofs)
__global__ void k_adjoint_pre(int nn, double dt, const uint8_t* clamp, const double* minv, const double* vb,
                              double* ab, double* y) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * nn) return;
    const int c = t / nn, n = t % nn;
    if (clamp[n] & (1 << c)) { y[t] = 0.0; ab[t] = 0.0; return; }
    const double a = fma(0.5 * dt, vb[t], ab[t]);
    ab[t] = a;
    y[t] = -a * minv[n];
}

// ubar' += VJP (gathered from the element buffer in a fixed order); then the adjoints at the previous
// step:  abar = dt/2 vbar' + dt^2/2 ubar',  vbar = vbar' + dt ubar',  ubar = ubar'
__global__ void k_adjoint_post(int nx, int ny, int nz, double dt, const uint8_t* clamp, const double* fe, double* ub,
                               double* vb, double* ab) {
    const int nn = (nx + 1) * (ny + 1) * (nz + 1);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * nn) return;
    const int c = t / nn, n = t % nn;
    if (clamp[n] & (1 << c)) { ub[t] = 0.0; vb[t] = 0.0; ab[t] = 0.0; return; }
    const int i = n % (nx + 1), q = n / (nx + 1);
    const double g = hex8::gather_force(fe, nx, ny, nz, nx * ny * nz, i, q % (ny + 1), q / (ny + 1), c);
    const double u = ub[t] + g;
    const double v = vb[t];
    ub[t] = u;
    ab[t] = fma(0.5 * dt * dt, u, 0.5 * dt * v);
    vb[t] = fma(dt, u, v);
}

}  // namespace

cudaError_t launch_adjoint_pre(int nn, double dt, const uint8_t* clamp, const double* minv, const double* vb, double* ab,
                               double* y, cudaStream_t s) {
    k_adjoint_pre<<<grid_for(3LL * nn, 256), 256, 0, s>>>(nn, dt, clamp, minv, vb, ab, y);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_post(int nx, int ny, int nz, double dt, const uint8_t* clamp, const double* fe, double* ub,
                                double* vb, double* ab, cudaStream_t s) {
    const long long nn = (long long)(nx + 1) * (ny + 1) * (nz + 1);
    k_adjoint_post<<<grid_for(3 * nn, 256), 256, 0, s>>>(nx, ny, nz, dt, clamp, fe, ub, vb, ab);
    return cudaGetLastError();
}

}  // namespace osam
