// Directional derivative of the Neo-Hookean first Piola-Kirchhoff stress (Appendix A.3, cofactor
// form P = beta cof(F) + alpha F): dP = (dP/dF)[G].  Shared by the force VJP of the adjoint and the
// tangent action of the implicit Newton solves (the tangent has major symmetry, so both are the same
// contraction).
//   dJ = cof(F) : G,  d trC = 2 F : G,  d alpha = -2/3 alpha dJ / J,
//   d beta = [kappa J dJ - 1/3 (d alpha trC + alpha d trC)] / J - beta dJ / J,
//   dP = d beta cof + beta dcof[G] + d alpha F + alpha G,  dcof linear in G (cof is quadratic in F).
#pragma once

#include <cuda_runtime.h>

#include "hex8_math.cuh"

namespace osam {
namespace tangent {

// dP = tangent(H)[G] with pre-scaled (kap2, mu, mu3); pk, pm = P_kappa : G, P_mu : G (unscaled params).
// With s = J^-1/3 (the force's reciprocal cube root), r3 = s^2 = J^-2/3 and invJ = s^3 = 1/J:
//   alpha = mu r3,  beta = kap2 (J - invJ) - mu3 r3 invJ trC,
//   dalpha = -2/3 alpha invJ dJ,  dbeta = invJ [(2 kap2 J - beta) dJ - 1/3 (dalpha trC + 2 alpha F:G)],
//   pk = 1/2 (J - invJ) dJ,  pm = r3 F:G - 1/3 r3 invJ trC dJ
// (no divisions: the thirds are multiplications by a rounded 1/3).
__device__ __forceinline__ void nh_tangent(const double H[3][3], const double G[3][3], double kap2, double mu,
                                           double mu3, double dP[3][3], double& pk, double& pm) {
    constexpr double third = 1.0 / 3.0;
    double F[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) F[i][j] = H[i][j] + (i == j ? 1.0 : 0.0);
    double cf[3][3], dc[3][3];
    cf[0][0] = fma(F[1][1], F[2][2], -F[1][2] * F[2][1]);
    cf[0][1] = fma(F[1][2], F[2][0], -F[1][0] * F[2][2]);
    cf[0][2] = fma(F[1][0], F[2][1], -F[1][1] * F[2][0]);
    cf[1][0] = fma(F[0][2], F[2][1], -F[0][1] * F[2][2]);
    cf[1][1] = fma(F[0][0], F[2][2], -F[0][2] * F[2][0]);
    cf[1][2] = fma(F[0][1], F[2][0], -F[0][0] * F[2][1]);
    cf[2][0] = fma(F[0][1], F[1][2], -F[0][2] * F[1][1]);
    cf[2][1] = fma(F[0][2], F[1][0], -F[0][0] * F[1][2]);
    cf[2][2] = fma(F[0][0], F[1][1], -F[0][1] * F[1][0]);
    dc[0][0] = fma(G[1][1], F[2][2], fma(F[1][1], G[2][2], -fma(G[1][2], F[2][1], F[1][2] * G[2][1])));
    dc[0][1] = fma(G[1][2], F[2][0], fma(F[1][2], G[2][0], -fma(G[1][0], F[2][2], F[1][0] * G[2][2])));
    dc[0][2] = fma(G[1][0], F[2][1], fma(F[1][0], G[2][1], -fma(G[1][1], F[2][0], F[1][1] * G[2][0])));
    dc[1][0] = fma(G[0][2], F[2][1], fma(F[0][2], G[2][1], -fma(G[0][1], F[2][2], F[0][1] * G[2][2])));
    dc[1][1] = fma(G[0][0], F[2][2], fma(F[0][0], G[2][2], -fma(G[0][2], F[2][0], F[0][2] * G[2][0])));
    dc[1][2] = fma(G[0][1], F[2][0], fma(F[0][1], G[2][0], -fma(G[0][0], F[2][1], F[0][0] * G[2][1])));
    dc[2][0] = fma(G[0][1], F[1][2], fma(F[0][1], G[1][2], -fma(G[0][2], F[1][1], F[0][2] * G[1][1])));
    dc[2][1] = fma(G[0][2], F[1][0], fma(F[0][2], G[1][0], -fma(G[0][0], F[1][2], F[0][0] * G[1][2])));
    dc[2][2] = fma(G[0][0], F[1][1], fma(F[0][0], G[1][1], -fma(G[0][1], F[1][0], F[0][1] * G[1][0])));
    const double J = fma(F[0][0], cf[0][0], fma(F[0][1], cf[0][1], F[0][2] * cf[0][2]));
    double trC = F[0][0] * F[0][0], dJ = cf[0][0] * G[0][0], FG = F[0][0] * G[0][0];
#pragma unroll
    for (int a = 1; a < 9; ++a) {
        const int i = a / 3, j = a % 3;
        trC = fma(F[i][j], F[i][j], trC);
        dJ = fma(cf[i][j], G[i][j], dJ);
        FG = fma(F[i][j], G[i][j], FG);
    }
    const double s = hex8::rcbrtT(J);
    const double r3 = s * s, invJ = r3 * s;
    const double alpha = mu * r3;
    const double beta = fma(-(mu3 * r3) * invJ, trC, kap2 * (J - invJ));
    const double dalpha = (-2.0 * third) * (alpha * invJ) * dJ;
    const double dB = third * fma(dalpha, trC, 2.0 * alpha * FG);
    const double dbeta = invJ * fma(fma(2.0 * kap2, J, -beta), dJ, -dB);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            dP[i][j] = fma(dbeta, cf[i][j], fma(beta, dc[i][j], fma(dalpha, F[i][j], alpha * G[i][j])));
    pk = 0.5 * (J - invJ) * dJ;
    pm = fma(r3, FG, -(third * r3 * invJ * trC) * dJ);
}

}  // namespace tangent
}  // namespace osam
