// Device-side arithmetic of the hex8 internal force, shared by the element-level kernels and the
// batched per-step kernels.
//
// Internal-force formulation (uniform cubic elements of edge h).  With unit-cube coordinates s,
// grad_X N = grad_s N / h, detJ * w = h^3/8 at each of the 8 Gauss points s = (1 -+ 1/sqrt3)/2, so
//   H = grad u = sum_a (u_a / h) (x) grad_s N_a,     f_a = (h^2/8) sum_gp P(H) grad_s N_a.
// Trilinear shape functions factor per axis, so both sums are evaluated by sum factorisation:
// edge differences along one axis followed by linear interpolation along the other two, 16 FP64
// operations per (component, direction) instead of 8 x 8; the transposed interpolation and the
// nodal sums run in the sum / difference (Walsh) basis of the 8 corners (element_force_grad).
// The Neo-Hookean stress of Appendix A.3, P = F S with
//   S = 1/2 kappa (det C - 1) C^-1 + mu (det C)^-1/3 (I - 1/3 tr C C^-1),
// is evaluated through F C^-1 = F^-T = cof(F) / J, i.e.
//   P = alpha F + beta cof(F),  alpha = mu J^-2/3,
//   beta = [1/2 kappa (J^2 - 1) - 1/3 mu J^-2/3 tr C] / J = 1/2 kappa (J - 1/J) - (1/3 mu J^-2/3 / J) tr C,
// with J^-1/3 from a reciprocal cube root, J^-2/3 = (J^-1/3)^2 and 1/J = (J^-1/3)^3 (no division).  At
// F = I the volumetric term vanishes exactly (J - 1/J = 0), so the stress there is mu - 3 (mu/3) rounded.
#pragma once

#include <cuda_runtime.h>

#include "fp_bits.cuh"
#include "osam.h"

namespace osam {
namespace hex8 {

constexpr double kG0 = 0.21132486540518711775;   // (1 - 1/sqrt(3)) / 2
constexpr double kG1 = 0.78867513459481288225;   // (1 + 1/sqrt(3)) / 2
constexpr double kGd = 0.57735026918962576451;   // kG1 - kG0 = 1/sqrt(3)

__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }

// x^(-1/3) in FP64 (x != 0): a single-precision seed y, then one third-order correction from the
// binomial series of the exact factor (1 - e)^(-1/3) = 1 + e/3 + 2e^2/9 + ..., e = 1 - x y^3 the seed's
// residual (Householder's third-order iteration for y^-3 = x).  The remaining error is ~14 e^3 / 81:
// with the seed's |e| < 1e-6 that is below the FP64 rounding.  Six FP64 operations; the seed's
// conversions are integer operations (f32_rz, f64_of).  Zero, Inf or NaN propagate to a non-finite
// result (caught by the step's criterion).
__device__ __forceinline__ double rcbrtT(double x) {
    const double y = f64_of(rcbrtf(f32_rz(x)));
    const double e = fma(-x, y * y * y, 1.0);
    return fma(y, e * fma(e, 2.0 / 9.0, 1.0 / 3.0), y);
}
__device__ __forceinline__ float rcbrtT(float x) { return rcbrtf(x); }

// nodal values D[b][e] on a unit square -> values at the 2x2 Gauss points out[q][r]; plus_one adds 1
// to every output (folded into the first stage: the weights of each stage sum to 1)
template <typename T>
__device__ __forceinline__ void lerp2(const T D[2][2], T out[2][2], bool plus_one = false) {
    T E[2][2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        T d = D[1][e] - D[0][e];
        const T base = plus_one ? D[0][e] + T(1) : D[0][e];
        E[0][e] = fmaT(T(kG0), d, base);
        E[1][e] = fmaT(T(kG1), d, base);
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        T d = E[q][1] - E[q][0];
        out[q][0] = fmaT(T(kG0), d, E[q][0]);
        out[q][1] = fmaT(T(kG1), d, E[q][0]);
    }
}

// transpose of lerp2: Gauss-point values S[q][r] -> nodal out[b][e] = sum l_b(g_q) l_e(g_r) S[q][r]
template <typename T>
__device__ __forceinline__ void lerp2T(const T S[2][2], T out[2][2]) {
    T V[2][2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        T s = S[q][0] + S[q][1];
        V[q][0] = fmaT(T(kGd), S[q][0], T(kG0) * s);  // g1 S0 + g0 S1
        V[q][1] = s - V[q][0];                        // g0 S0 + g1 S1
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        T s = V[0][e] + V[1][e];
        out[0][e] = fmaT(T(kGd), V[0][e], T(kG0) * s);
        out[1][e] = s - out[0][e];
    }
}

// Appendix A.1: P = lambda tr(eps) I + 2 mu eps (lam, mu pre-scaled by h^2/8)
template <typename T>
__device__ __forceinline__ void stress_le(const T H[3][3], T lam, T mu, T P[3][3]) {
    T lt = lam * (H[0][0] + H[1][1] + H[2][2]);
    T mu2 = mu + mu;
#pragma unroll
    for (int c = 0; c < 3; ++c) P[c][c] = fmaT(mu2, H[c][c], lt);
    P[0][1] = P[1][0] = mu * (H[0][1] + H[1][0]);
    P[0][2] = P[2][0] = mu * (H[0][2] + H[2][0]);
    P[1][2] = P[2][1] = mu * (H[1][2] + H[2][1]);
}

// Appendix A.2 Saint Venant-Kirchhoff (lam, mu pre-scaled by h^2/8): E = 1/2 (H + H^T + H^T H),
// S = lam tr(E) I + 2 mu E, P = (I + H) S
template <typename T>
__device__ __forceinline__ void stress_svk(const T H[3][3], T lam, T mu, T P[3][3]) {
    T S[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            T c = H[i][j] + H[j][i];
#pragma unroll
            for (int k = 0; k < 3; ++k) c = fmaT(H[k][i], H[k][j], c);
            S[i][j] = T(0.5) * c;  // E
        }
    const T lt = lam * (S[0][0] + S[1][1] + S[2][2]);
    const T mu2 = mu + mu;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            S[i][j] = i == j ? fmaT(mu2, S[i][j], lt) : mu2 * S[i][j];
            if (j != i) S[j][i] = S[i][j];
        }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T p = S[i][j];
#pragma unroll
            for (int k = 0; k < 3; ++k) p = fmaT(H[i][k], S[k][j], p);
            P[i][j] = p;
        }
}

// Material factors (m1, m2, m3) of element_force_grad: Neo-Hookean (kappa/2, mu, mu/3) or linear
// elastic / Saint Venant-Kirchhoff (lambda, mu, 0), each times wq = h^2/32 -- the Gauss weight times
// detJ / h (h^2/8) and the 1/4 of the Walsh-basis transposed interpolation.  wq3 = wq / 3.
template <int MAT, typename T>
__device__ __forceinline__ void material_factors(double lam, double mu, double wq, double wq3, T& m1, T& m2, T& m3) {
    if (MAT == OSAM_NEO_HOOKEAN) {
        const double kappa = lam + (2.0 / 3.0) * mu;
        m1 = T(0.5 * kappa * wq); m2 = T(mu * wq); m3 = T(mu * wq3);
    } else {
        m1 = T(lam * wq); m2 = T(mu * wq); m3 = T(0);
    }
}

// Appendix A.3 in cofactor form (kap2 = kappa/2, mu, mu3 = mu/3, all pre-scaled by h^2/8):
// P = alpha F + beta cof(F); returns F, cof(F), alpha, beta
template <typename T>
__device__ __forceinline__ void nh_factors(const T H[3][3], T kap2, T mu, T mu3, T F[3][3], T C[3][3], T& alpha,
                                           T& beta) {
    F[0][0] = T(1) + H[0][0]; F[1][1] = T(1) + H[1][1]; F[2][2] = T(1) + H[2][2];
    F[0][1] = H[0][1]; F[0][2] = H[0][2]; F[1][0] = H[1][0]; F[1][2] = H[1][2]; F[2][0] = H[2][0]; F[2][1] = H[2][1];
    C[0][0] = fmaT(F[1][1], F[2][2], -F[1][2] * F[2][1]);
    C[0][1] = fmaT(F[1][2], F[2][0], -F[1][0] * F[2][2]);
    C[0][2] = fmaT(F[1][0], F[2][1], -F[1][1] * F[2][0]);
    C[1][0] = fmaT(F[0][2], F[2][1], -F[0][1] * F[2][2]);
    C[1][1] = fmaT(F[0][0], F[2][2], -F[0][2] * F[2][0]);
    C[1][2] = fmaT(F[0][1], F[2][0], -F[0][0] * F[2][1]);
    C[2][0] = fmaT(F[0][1], F[1][2], -F[0][2] * F[1][1]);
    C[2][1] = fmaT(F[0][2], F[1][0], -F[0][0] * F[1][2]);
    C[2][2] = fmaT(F[0][0], F[1][1], -F[0][1] * F[1][0]);
    const T J = fmaT(F[0][0], C[0][0], fmaT(F[0][1], C[0][1], F[0][2] * C[0][2]));
    T trC = F[0][0] * F[0][0];
#pragma unroll
    for (int k = 1; k < 9; ++k) trC = fmaT(F[k / 3][k % 3], F[k / 3][k % 3], trC);
    const T s1 = rcbrtT(J);                  // J^-1/3
    const T r3 = s1 * s1;                    // J^-2/3
    const T invJ = r3 * s1;                  // 1/J
    alpha = mu * r3;
    beta = fmaT(-(mu3 * r3) * invJ, trC, kap2 * (J - invJ));
}

template <typename T>
__device__ __forceinline__ void stress_nh(const T H[3][3], T kap2, T mu, T mu3, T P[3][3]) {
    T F[3][3], C[3][3], alpha, beta;
    nh_factors<T>(H, kap2, mu, mu3, F, C, alpha, beta);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) P[i][j] = fmaT(alpha, F[i][j], beta * C[i][j]);
}

// Neo-Hookean Gauss-point sums Sx[c][q][r] = sum_p P_c0(p, q, r), Sy[c][p][r] = sum_q P_c1,
// Sz[c][p][q] = sum_r P_c2 with P = alpha F + beta cof(F).  The inputs are the columns of F = I + H at
// the Gauss points: Gx = dx u + e_x, Gy = dy u + e_y, Gz = dz u + e_z (the callers add the 1 of the
// diagonal before the last interpolation stage, where it costs fewer operations; rigid translations
// still give F = I exactly).  Column k of F depends on two of the three
// Gauss indices only (column 0 on q and r, column 1 on p and r, column 2 on p and q), so
//  - tr C = |F_0|^2 + |F_1|^2 + |F_2|^2 is assembled from squared column norms formed once per pair of
//    Gauss points that share the column, and
//  - in each sum the alpha F term of a pair is one product (alpha_a + alpha_b) F_k,
// which takes ~50 FP64 operations per element off the one-Gauss-point-at-a-time evaluation.
// `at_gp(p, q, r, F, cofF, J, trC, invJ, alpha, beta)` is called at every Gauss point with its
// quantities (the implicit Newton force stores them as the tangent's linearisation); the default
// does nothing and compiles away.
struct NoGaussHook {
    template <typename T>
    __device__ __forceinline__ void operator()(int, int, int, const T (&)[3][3], const T (&)[3][3], T, T, T, T,
                                               T) const {}
};

template <typename T, typename Hook = NoGaussHook>
__device__ __forceinline__ void nh_gauss_sums(const T Gx[3][2][2], const T Gy[3][2][2], const T Gz[3][2][2],
                                              T kap2, T mu, T mu3, T Sx[3][2][2], T Sy[3][2][2], T Sz[3][2][2],
                                              const Hook& at_gp = Hook()) {
    const T (*F0)[2][2] = Gx;   // columns of F: F0[c][q][r], F1[c][p][r], F2[c][p][q]
    const T (*F1)[2][2] = Gy;
    const T (*F2)[2][2] = Gz;
    T n0[2][2];                                // |F_0|^2 at (q, r)
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int r = 0; r < 2; ++r)
            n0[q][r] = fmaT(F0[2][q][r], F0[2][q][r], fmaT(F0[1][q][r], F0[1][q][r], F0[0][q][r] * F0[0][q][r]));
    T ax[2][2];                                // alpha at (0, q, r), waiting for its pair (1, q, r)
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        T n1[2], n2[2];                        // |F_1|^2 at (p, r), |F_2|^2 at (p, q)
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            n1[a] = fmaT(F1[2][p][a], F1[2][p][a], fmaT(F1[1][p][a], F1[1][p][a], F1[0][p][a] * F1[0][p][a]));
            n2[a] = fmaT(F2[2][p][a], F2[2][p][a], fmaT(F2[1][p][a], F2[1][p][a], F2[0][p][a] * F2[0][p][a]));
        }
        T ay[2];                               // alpha at (p, 0, r)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            T az = T(0);                       // alpha at (p, q, 0)
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                T Fm[3][3], Cm[3][3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    Fm[c][0] = F0[c][q][r];
                    Fm[c][1] = F1[c][p][r];
                    Fm[c][2] = F2[c][p][q];
                }
                Cm[0][0] = fmaT(Fm[1][1], Fm[2][2], -Fm[1][2] * Fm[2][1]);
                Cm[0][1] = fmaT(Fm[1][2], Fm[2][0], -Fm[1][0] * Fm[2][2]);
                Cm[0][2] = fmaT(Fm[1][0], Fm[2][1], -Fm[1][1] * Fm[2][0]);
                Cm[1][0] = fmaT(Fm[0][2], Fm[2][1], -Fm[0][1] * Fm[2][2]);
                Cm[1][1] = fmaT(Fm[0][0], Fm[2][2], -Fm[0][2] * Fm[2][0]);
                Cm[1][2] = fmaT(Fm[0][1], Fm[2][0], -Fm[0][0] * Fm[2][1]);
                Cm[2][0] = fmaT(Fm[0][1], Fm[1][2], -Fm[0][2] * Fm[1][1]);
                Cm[2][1] = fmaT(Fm[0][2], Fm[1][0], -Fm[0][0] * Fm[1][2]);
                Cm[2][2] = fmaT(Fm[0][0], Fm[1][1], -Fm[0][1] * Fm[1][0]);
                const T J = fmaT(Fm[0][0], Cm[0][0], fmaT(Fm[0][1], Cm[0][1], Fm[0][2] * Cm[0][2]));
                const T trC = (n0[q][r] + n1[r]) + n2[q];
                const T s1 = rcbrtT(J);        // J^-1/3
                const T r3 = s1 * s1;          // J^-2/3
                const T invJ = r3 * s1;        // 1/J
                const T alpha = mu * r3;
                const T beta = fmaT(-(mu3 * r3) * invJ, trC, kap2 * (J - invJ));
                at_gp(p, q, r, Fm, Cm, J, trC, invJ, alpha, beta);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    Sx[c][q][r] = p == 0 ? beta * Cm[c][0] : fmaT(beta, Cm[c][0], Sx[c][q][r]);
                    Sy[c][p][r] = q == 0 ? beta * Cm[c][1] : fmaT(beta, Cm[c][1], Sy[c][p][r]);
                    Sz[c][p][q] = r == 0 ? beta * Cm[c][2] : fmaT(beta, Cm[c][2], Sz[c][p][q]);
                }
                if (p == 0) {
                    ax[q][r] = alpha;
                } else {
                    const T a = ax[q][r] + alpha;
#pragma unroll
                    for (int c = 0; c < 3; ++c) Sx[c][q][r] = fmaT(a, Fm[c][0], Sx[c][q][r]);
                }
                if (q == 0) {
                    ay[r] = alpha;
                } else {
                    const T a = ay[r] + alpha;
#pragma unroll
                    for (int c = 0; c < 3; ++c) Sy[c][p][r] = fmaT(a, Fm[c][1], Sy[c][p][r]);
                }
                if (r == 0) {
                    az = alpha;
                } else {
                    const T a = az + alpha;
#pragma unroll
                    for (int c = 0; c < 3; ++c) Sz[c][p][q] = fmaT(a, Fm[c][2], Sz[c][p][q]);
                }
            }
        }
    }
}

// Hadamard (sum / difference) coefficients of a 2x2 array S[a][b]: h0 = sum, ha = sum (2a - 1) S,
// hb = sum (2b - 1) S, hab = sum (2a - 1)(2b - 1) S (two butterfly stages, 8 additions)
template <typename T>
__device__ __forceinline__ void hadamard2(const T S[2][2], T& h0, T& ha, T& hb, T& hab) {
    const T e0 = S[0][0] + S[0][1], e1 = S[1][0] + S[1][1];
    const T d0 = S[0][1] - S[0][0], d1 = S[1][1] - S[1][0];
    h0 = e0 + e1; ha = e1 - e0; hb = d0 + d1; hab = d1 - d0;
}

template <typename T>
__device__ __forceinline__ void walsh_transpose(const T Sx[3][2][2], const T Sy[3][2][2], const T Sz[3][2][2],
                                                T F[3][8]);

// Element force from the displacement gradients at the Gauss points:
//   Gx[c][q][r] = d u_c / dx at (y GP q, z GP r), Gy[c][p][r], Gz[c][p][q]
// (Neo-Hookean: the columns of F, i.e. with the 1 of the diagonal added, see nh_gauss_sums), and the
// material factors of material_factors().  Output F[c][corner], corner = ax + 2 ay + 4 az.
//
// Transposed interpolation in the Walsh basis.  With s_d = 2 a_d - 1 the sign of a corner along axis d
// and t = 1/sqrt3, the trilinear weights at the Gauss points are l_a(g_q) = (1 + s t_q) / 2 with
// t_q = (2q - 1) t, so the force of the x-direction sums Sx[q][r] at corner s is
//   s_x Tx = s_x / 4 [h0(Sx) + t s_y ha(Sx) + t s_z hb(Sx) + t^2 s_y s_z hab(Sx)],
// and likewise for y and z.  Summed over the directions, the corner force is
//   F(s) = 1/4 [wx sx + wy sy + wz sz + t (wxy sx sy + wxz sx sz + wyz sy sz) + t^2 wxyz sx sy sz],
//   wx = h0(Sx), wy = h0(Sy), wz = h0(Sz), wxy = ha(Sx) + ha(Sy), wxz = hb(Sx) + ha(Sz),
//   wyz = hb(Sy) + hb(Sz), wxyz = hab(Sx) + hab(Sy) + hab(Sz)
// (no constant term: the element force is self-equilibrated).  With P = sx wx + sy wy + t sx sy wxy
// and Q = wz + t sx wxz + t sy wyz + t^2 sx sy wxyz, F = (P + sz Q) / 4; the 1/4 is in the material
// factors.  51 FP64 operations per component instead of 64 for three tensor-product transposes.
template <int MAT, typename T>
__device__ __forceinline__ void element_force_grad(const T Gx[3][2][2], const T Gy[3][2][2], const T Gz[3][2][2],
                                                   T m1, T m2, T m3, T F[3][8]) {
    T Sx[3][2][2], Sy[3][2][2], Sz[3][2][2];
    if constexpr (MAT == OSAM_NEO_HOOKEAN) {
        nh_gauss_sums<T>(Gx, Gy, Gz, m1, m2, m3, Sx, Sy, Sz);
    } else {
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int q = 0; q < 2; ++q)
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    T Hm[3][3], P[3][3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        Hm[c][0] = Gx[c][q][r];
                        Hm[c][1] = Gy[c][p][r];
                        Hm[c][2] = Gz[c][p][q];
                    }
                    if (MAT == OSAM_SAINT_VENANT_KIRCHHOFF) stress_svk<T>(Hm, m1, m2, P);
                    else stress_le<T>(Hm, m1, m2, P);
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        if (p == 0) Sx[c][q][r] = P[c][0]; else Sx[c][q][r] += P[c][0];
                        if (q == 0) Sy[c][p][r] = P[c][1]; else Sy[c][p][r] += P[c][1];
                        if (r == 0) Sz[c][p][q] = P[c][2]; else Sz[c][p][q] += P[c][2];
                    }
                }
    }
    walsh_transpose<T>(Sx, Sy, Sz, F);
}

// The transposed interpolation and nodal sums of element_force_grad on its own (Gauss-point sums S
// scaled by 1/4 -> corner forces F[c][corner]); also used by the force's vector-Jacobian product.
template <typename T>
__device__ __forceinline__ void walsh_transpose(const T Sx[3][2][2], const T Sy[3][2][2], const T Sz[3][2][2],
                                                T F[3][8]) {
    const T t = T(kGd);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        T wx, ax_, bx_, abx, wy, ay_, by_, aby, wz, az_, bz_, abz;
        hadamard2<T>(Sx[c], wx, ax_, bx_, abx);   // Sx[q][r]: a along y, b along z
        hadamard2<T>(Sy[c], wy, ay_, by_, aby);   // Sy[p][r]: a along x, b along z
        hadamard2<T>(Sz[c], wz, az_, bz_, abz);   // Sz[p][q]: a along x, b along y
        const T wxy = ax_ + ay_, wxz = bx_ + az_, wyz = by_ + bz_, wxyz = (abx + aby) + abz;
        const T up = fmaT(t, wxy, wx), um = fmaT(-t, wxy, wx);      // wx + t sy wxy, sy = +1 / -1
        const T ap = fmaT(t, wyz, wz), am = fmaT(-t, wyz, wz);      // wz + t sy wyz
        const T bp = fmaT(t, wxyz, wxz), bm = fmaT(-t, wxyz, wxz);  // wxz + t sy wxyz
        // P and Q at (sx, sy) = (+,+), (-,+), (+,-), (-,-); corner index ax + 2 ay + 4 az
        const T Ppp = up + wy, Pmp = wy - up, Ppm = um - wy, Pmm = -um - wy;
        const T Qpp = fmaT(t, bp, ap), Qmp = fmaT(-t, bp, ap), Qpm = fmaT(t, bm, am), Qmm = fmaT(-t, bm, am);
        F[c][3] = Ppp - Qpp; F[c][7] = Ppp + Qpp;
        F[c][2] = Pmp - Qmp; F[c][6] = Pmp + Qmp;
        F[c][1] = Ppm - Qpm; F[c][5] = Ppm + Qpm;
        F[c][0] = Pmm - Qmm; F[c][4] = Pmm + Qmm;
    }
}

// Element force from scaled edge differences.
//   Dx[c][ay][az] = (u_c(1,ay,az) - u_c(0,ay,az)) / h   (and Dy[c][ax][az], Dz[c][ax][ay])
template <int MAT, typename T>
__device__ __forceinline__ void element_force(const T Dx[3][2][2], const T Dy[3][2][2], const T Dz[3][2][2],
                                              T m1, T m2, T m3, T F[3][8]) {
    T Gx[3][2][2], Gy[3][2][2], Gz[3][2][2];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const bool nh = MAT == OSAM_NEO_HOOKEAN;
        lerp2<T>(Dx[c], Gx[c], nh && c == 0);   // Gx[c][q][r]  (q: y Gauss point, r: z Gauss point)
        lerp2<T>(Dy[c], Gy[c], nh && c == 1);   // Gy[c][p][r]
        lerp2<T>(Dz[c], Gz[c], nh && c == 2);   // Gz[c][p][q]
    }
    element_force_grad<MAT, T>(Gx, Gy, Gz, m1, m2, m3, F);
}

__device__ __forceinline__ void atomic_add(double* p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void atomic_add(float* p, float v) { atomicAdd(p, v); }

// scaled edge differences of the 8 nodal values of one component (FP64 arithmetic, T output)
template <typename T>
__device__ __forceinline__ void edge_differences(const double U[8], double invh, T Dx[2][2], T Dy[2][2], T Dz[2][2]) {
    if constexpr (sizeof(T) == 8) {
        double V[8];
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8) V[c8] = U[c8] * invh;
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                Dx[p][q] = T(V[1 + 2 * p + 4 * q] - V[2 * p + 4 * q]);
                Dy[p][q] = T(V[p + 2 + 4 * q] - V[p + 4 * q]);
                Dz[p][q] = T(V[p + 2 * q + 4] - V[p + 2 * q]);
            }
    } else {
        // FP32 force: differences in FP64 (they cancel), the rest in FP32
        const float ih = float(invh);
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                Dx[p][q] = T(U[1 + 2 * p + 4 * q] - U[2 * p + 4 * q]) * ih;
                Dy[p][q] = T(U[p + 2 + 4 * q] - U[p + 4 * q]) * ih;
                Dz[p][q] = T(U[p + 2 * q + 4] - U[p + 2 * q]) * ih;
            }
    }
}

// edge differences of nodal values already divided by h (the batched kernels read the displacement
// copy u/h that the node kernel writes with the predictor, saving 24 multiplications per element)
template <typename T>
__device__ __forceinline__ void edge_differences_prescaled(const double V[8], T Dx[2][2], T Dy[2][2], T Dz[2][2]) {
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            Dx[p][q] = T(V[1 + 2 * p + 4 * q] - V[2 * p + 4 * q]);
            Dy[p][q] = T(V[p + 2 + 4 * q] - V[p + 4 * q]);
            Dz[p][q] = T(V[p + 2 * q + 4] - V[p + 2 * q]);
        }
}

// edge differences for the FP32 force from the (hi, lo) float split of u/h (hi = fl32(u/h), lo =
// fl32(u/h - hi)): (hi1 - hi0) + (lo1 - lo0) on the FP32 pipes.  For neighbouring nodes of a smooth
// field hi1 - hi0 is exact (Sterbenz) or far larger than the lo terms, so the difference keeps FP32
// relative accuracy without FP64 arithmetic (the FP64 form costs an FP64 subtraction and conversion
// per difference, which bound the FP32 kernel by the FP64 pipe).
__device__ __forceinline__ void edge_differences_split(const float2 V[8], float Dx[2][2], float Dy[2][2],
                                                       float Dz[2][2]) {
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const float2 x1 = V[1 + 2 * p + 4 * q], x0 = V[2 * p + 4 * q];
            const float2 y1 = V[p + 2 + 4 * q], y0 = V[p + 4 * q];
            const float2 z1 = V[p + 2 * q + 4], z0 = V[p + 2 * q];
            Dx[p][q] = (x1.x - x0.x) + (x1.y - x0.y);
            Dy[p][q] = (y1.x - y0.x) + (y1.y - y0.y);
            Dz[p][q] = (z1.x - z0.x) + (z1.y - z0.y);
        }
}

// (hi, lo) float split of an FP64 value for the FP32 force: hi = v cut to 24 bits, lo = the exact
// remainder v - hi cut to 24 bits (|v - (hi + lo)| < 2^-47 |v|), by integer conversions
__device__ __forceinline__ float2 split_f2(double v) {
    const float hi = f32_rz(v);
    return make_float2(hi, f32_rz(v - f64_of(hi)));
}

// nodal force of node (i,j,k), component c, from the element buffer (fixed order: deterministic)
template <typename TF>
__device__ __forceinline__ double gather_force(const TF* fe, int nx, int ny, int nz, int ne, int i, int j, int k,
                                               int c) {
    double s = 0.0;
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
                const int e = ie + nx * (je + ny * ke);
                const int corner = ax + 2 * ay + 4 * az;
                s += double(fe[(long long)(corner * 3 + c) * ne + e]);
            }
        }
    }
    return s;
}

}  // namespace hex8
}  // namespace osam
