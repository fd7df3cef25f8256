// Directional derivative of the Neo-Hookean first Piola-Kirchhoff stress (Appendix A.3, cofactor
// form P = beta cof(F) + alpha F): dP = (dP/dF)[G].  Shared by the force VJP of the adjoint and the
// tangent action of the implicit Newton solves (the tangent has major symmetry, so both are the same
// contraction).
//   dJ = cof(F) : G,  d trC = 2 F : G,  d alpha = -2/3 alpha dJ / J,
//   d beta = [kappa J dJ - 1/3 (d alpha trC + alpha d trC)] / J - beta dJ / J,
//   dP = d beta cof + beta dcof[G] + d alpha F + alpha G,  dcof linear in G (cof is quadratic in F).
#pragma once

#include <cuda_runtime.h>

namespace osam {
namespace tangent {

// dP = tangent(H)[G] with pre-scaled (kap2, mu, mu3); pk, pm = P_kappa : G, P_mu : G (unscaled params)
__device__ __forceinline__ void nh_tangent(const double H[3][3], const double G[3][3], double kap2, double mu,
                                           double mu3, double dP[3][3], double& pk, double& pm) {
    double F[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) F[i][j] = H[i][j] + (i == j ? 1.0 : 0.0);
    double cf[3][3], dc[3][3];
    cf[0][0] = F[1][1] * F[2][2] - F[1][2] * F[2][1];
    cf[0][1] = F[1][2] * F[2][0] - F[1][0] * F[2][2];
    cf[0][2] = F[1][0] * F[2][1] - F[1][1] * F[2][0];
    cf[1][0] = F[0][2] * F[2][1] - F[0][1] * F[2][2];
    cf[1][1] = F[0][0] * F[2][2] - F[0][2] * F[2][0];
    cf[1][2] = F[0][1] * F[2][0] - F[0][0] * F[2][1];
    cf[2][0] = F[0][1] * F[1][2] - F[0][2] * F[1][1];
    cf[2][1] = F[0][2] * F[1][0] - F[0][0] * F[1][2];
    cf[2][2] = F[0][0] * F[1][1] - F[0][1] * F[1][0];
    dc[0][0] = G[1][1] * F[2][2] + F[1][1] * G[2][2] - G[1][2] * F[2][1] - F[1][2] * G[2][1];
    dc[0][1] = G[1][2] * F[2][0] + F[1][2] * G[2][0] - G[1][0] * F[2][2] - F[1][0] * G[2][2];
    dc[0][2] = G[1][0] * F[2][1] + F[1][0] * G[2][1] - G[1][1] * F[2][0] - F[1][1] * G[2][0];
    dc[1][0] = G[0][2] * F[2][1] + F[0][2] * G[2][1] - G[0][1] * F[2][2] - F[0][1] * G[2][2];
    dc[1][1] = G[0][0] * F[2][2] + F[0][0] * G[2][2] - G[0][2] * F[2][0] - F[0][2] * G[2][0];
    dc[1][2] = G[0][1] * F[2][0] + F[0][1] * G[2][0] - G[0][0] * F[2][1] - F[0][0] * G[2][1];
    dc[2][0] = G[0][1] * F[1][2] + F[0][1] * G[1][2] - G[0][2] * F[1][1] - F[0][2] * G[1][1];
    dc[2][1] = G[0][2] * F[1][0] + F[0][2] * G[1][0] - G[0][0] * F[1][2] - F[0][0] * G[1][2];
    dc[2][2] = G[0][0] * F[1][1] + F[0][0] * G[1][1] - G[0][1] * F[1][0] - F[0][1] * G[1][0];
    const double J = F[0][0] * cf[0][0] + F[0][1] * cf[0][1] + F[0][2] * cf[0][2];
    double trC = 0.0, dJ = 0.0, FG = 0.0, cG = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            trC += F[i][j] * F[i][j];
            dJ += cf[i][j] * G[i][j];
            FG += F[i][j] * G[i][j];
        }
    cG = dJ;
    const double dtrC = 2.0 * FG;
    const double J2 = J * J;
    const double r3 = rcbrt(J2);
    const double invJ = J * (r3 * r3 * r3);
    const double alpha = mu * r3;
    const double beta = (kap2 * (J2 - 1.0) - mu3 * r3 * trC) * invJ;
    const double dalpha = -(2.0 / 3.0) * alpha * dJ * invJ;
    const double dA = 2.0 * kap2 * J * dJ;
    const double dB = (dalpha * trC + alpha * dtrC) / 3.0;
    const double dbeta = (dA - dB) * invJ - beta * dJ * invJ;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) dP[i][j] = dbeta * cf[i][j] + beta * dc[i][j] + dalpha * F[i][j] + alpha * G[i][j];
    // P_kappa = 1/2 (J^2 - 1)/J cof ; P_mu = J^-2/3 F - 1/3 J^-2/3 trC / J cof
    pk = 0.5 * (J2 - 1.0) * invJ * cG;
    pm = r3 * FG - (r3 * trC * invJ / 3.0) * cG;
}

}  // namespace tangent
}  // namespace osam
