/*
 * osam_oracle.c -- plain, slow, FP64 CPU oracle of the O-SAM FOM / OpInf hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call this file:
 * only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs use it.
 * It shares no source, header, table or helper with the CUDA library.
 *
 * What it computes, each part written from the paper's statement of the method
 * (arXiv 2511.20687, "Hybrid coupling with operator inference and the overlapping Schwarz
 * alternating method"):
 *   - hex8 isoparametric internal force  f_int = sum_e sum_gp w detJ P(F) grad N   (Sec. 2, Eq. 5;
 *     2x2x2 Gauss, general Jacobian of every element, standard isoparametric FE)
 *   - constitutive laws of Appendix A: linear elastic (A.1) and Neo-Hookean (A.3).  The deviatoric
 *     coefficient of S is 1/3, obtained by differentiating the printed energy A_dev (the printed 1/2
 *     disagrees with that energy; tests pin P against finite differences of A).
 *   - row-sum lumped mass (each element gives rho*V_e/8 to each of its nodes; Sec. 5 setup)
 *   - explicit Newmark (beta = 0, gamma = 1/2) in predictor / corrector form (Sec. 4.1), and implicit
 *     Newmark (beta = 1/4, gamma = 1/2) solved by Newton's method with the exact tangent
 *   - O-SAM controller of Algorithm 1 / Eq. schwarz_discrete with the criterion conv_criterion:
 *     multiplicative sweep over the subdomains in index order (or the additive variant of Remark
 *     additive_sam: every subdomain from the previous iteration's data), pointwise spatial projector Pi
 *     (trilinear interpolation in a donor element found by brute-force search and Newton inversion
 *     of the trilinear map), temporal interpolant Xi linear between the source's time levels
 *     (identity when the time steps agree); each subdomain has its own number of substeps.
 *   - quadratic OpInf ROM subdomain of Eq. schwarz_opinf_discrete, written in the solved form
 *     qdd = K q + H kron_c(q) + B ghat + c, with ghat = Phi_S^T s (boundary POD, Sec. 4.2.1) and the
 *     ROM -> FOM trace Pi (Phi q) built from the reconstructed full field.
 *   - reverse-mode adjoint of the explicit rollout (hand derived; the NH tangent is the directional
 *     derivative of P = F S(C)).
 *
 * Every state vector is interleaved [node][3].  Node (i,j,k) of an nx*ny*nz element box has index
 * i + (nx+1)*(j + (ny+1)*k); element (i,j,k) has index i + nx*(j + ny*k).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_SUB 8
#define ORC_MAX_CPL 16

enum { ORC_OK = 0, ORC_MAXITER = 1, ORC_EINVAL = -1, ORC_ECFL = -2, ORC_ENONFINITE = -3, ORC_EDONOR = -4, ORC_ENOMEM = -7 };
enum { ORC_LE = 0, ORC_NH = 1, ORC_SVK = 2 };
enum { ORC_FOM = 0, ORC_ROM = 1 };

/* ------------------------------------------------------------------------------------------ */
/* mesh                                                                                        */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int nx, ny, nz;
    double h, org[3];
    int nn, ne;
} omesh;

static void mesh_set(omesh* m, int nx, int ny, int nz, double h, const double* org) {
    m->nx = nx; m->ny = ny; m->nz = nz; m->h = h;
    m->org[0] = org[0]; m->org[1] = org[1]; m->org[2] = org[2];
    m->nn = (nx + 1) * (ny + 1) * (nz + 1);
    m->ne = nx * ny * nz;
}

static void node_X(const omesh* m, int n, double X[3]) {
    int i = n % (m->nx + 1);
    int j = (n / (m->nx + 1)) % (m->ny + 1);
    int k = n / ((m->nx + 1) * (m->ny + 1));
    X[0] = m->org[0] + i * m->h;
    X[1] = m->org[1] + j * m->h;
    X[2] = m->org[2] + k * m->h;
}

/* reference corner signs of the 8 hex nodes, standard counter-clockwise order, bottom then top */
static const int CORNER[8][3] = {
    {-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
    {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};

static void elem_nodes(const omesh* m, int e, int nodes[8]) {
    int i = e % m->nx, j = (e / m->nx) % m->ny, k = e / (m->nx * m->ny);
    for (int a = 0; a < 8; ++a) {
        int ii = i + (CORNER[a][0] > 0), jj = j + (CORNER[a][1] > 0), kk = k + (CORNER[a][2] > 0);
        nodes[a] = ii + (m->nx + 1) * (jj + (m->ny + 1) * kk);
    }
}

/* trilinear shape functions and their reference gradients */
static void shape(const double xi[3], double N[8], double dN[8][3]) {
    for (int a = 0; a < 8; ++a) {
        double sx = CORNER[a][0], sy = CORNER[a][1], sz = CORNER[a][2];
        double fx = 1.0 + sx * xi[0], fy = 1.0 + sy * xi[1], fz = 1.0 + sz * xi[2];
        N[a] = 0.125 * fx * fy * fz;
        dN[a][0] = 0.125 * sx * fy * fz;
        dN[a][1] = 0.125 * fx * sy * fz;
        dN[a][2] = 0.125 * fx * fy * sz;
    }
}

static double det3(const double A[3][3]) {
    return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1])
         - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])
         + A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

static void inv3(const double A[3][3], double B[3][3]) {
    double d = det3(A);
    B[0][0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) / d;
    B[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / d;
    B[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / d;
    B[1][0] = (A[1][2] * A[2][0] - A[1][0] * A[2][2]) / d;
    B[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / d;
    B[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / d;
    B[2][0] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) / d;
    B[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / d;
    B[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / d;
}

/* Gauss point g of the 2x2x2 rule: xi = corner sign / sqrt(3), weight 1 */
static void gauss_point(int g, double xi[3]) {
    const double s = 1.0 / sqrt(3.0);
    xi[0] = CORNER[g][0] * s; xi[1] = CORNER[g][1] * s; xi[2] = CORNER[g][2] * s;
}

/* physical shape gradients dNdX[a][i] = dN_a/dX_i and detJ at Gauss point g of element nodes X */
static double physical_gradients(const double X[8][3], int g, double dNdX[8][3]) {
    double xi[3], N[8], dN[8][3], J[3][3], Ji[3][3];
    gauss_point(g, xi);
    shape(xi, N, dN);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            J[i][j] = 0.0;
            for (int a = 0; a < 8; ++a) J[i][j] += X[a][i] * dN[a][j];
        }
    inv3(J, Ji);
    for (int a = 0; a < 8; ++a)
        for (int i = 0; i < 3; ++i) {
            dNdX[a][i] = 0.0;
            for (int j = 0; j < 3; ++j) dNdX[a][i] += dN[a][j] * Ji[j][i];
        }
    return det3(J);
}

/* ------------------------------------------------------------------------------------------ */
/* constitutive laws, Appendix A                                                               */
/* ------------------------------------------------------------------------------------------ */
/* A.1 linear elastic: eps = sym(grad u), sigma = lambda tr(eps) I + 2 mu eps; P = sigma */
static void stress_le(const double H[3][3], double lam, double mu, double P[3][3]) {
    double eps[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) eps[i][j] = 0.5 * (H[i][j] + H[j][i]);
    double tr = eps[0][0] + eps[1][1] + eps[2][2];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) P[i][j] = 2.0 * mu * eps[i][j] + (i == j ? lam * tr : 0.0);
}

static double energy_le(const double H[3][3], double lam, double mu) {
    double eps[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) eps[i][j] = 0.5 * (H[i][j] + H[j][i]);
    double tr = eps[0][0] + eps[1][1] + eps[2][2], tr2 = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) tr2 += eps[i][j] * eps[j][i];
    return 0.5 * lam * tr * tr + mu * tr2;
}

/* A.3 Neo-Hookean: F = I + H, C = F^T F,
 *   S = 1/2 kappa (det C - 1) C^-1 + mu (det C)^(-1/3) (I - 1/3 tr(C) C^-1),  P = F S,
 * kappa = lambda + 2/3 mu (bulk modulus from the Lame pair). */
static void nh_parts(const double H[3][3], double Pk[3][3], double Pm[3][3]) {
    /* P = kappa * Pk + mu * Pm */
    double F[3][3], C[3][3], Ci[3][3], Sk[3][3], Sm[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) F[i][j] = H[i][j] + (i == j ? 1.0 : 0.0);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            C[i][j] = 0.0;
            for (int k = 0; k < 3; ++k) C[i][j] += F[k][i] * F[k][j];
        }
    double dC = det3(C);
    inv3(C, Ci);
    double trC = C[0][0] + C[1][1] + C[2][2];
    double g = pow(dC, -1.0 / 3.0);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            Sk[i][j] = 0.5 * (dC - 1.0) * Ci[i][j];
            Sm[i][j] = g * ((i == j ? 1.0 : 0.0) - trC * Ci[i][j] / 3.0);
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            Pk[i][j] = 0.0; Pm[i][j] = 0.0;
            for (int k = 0; k < 3; ++k) {
                Pk[i][j] += F[i][k] * Sk[k][j];
                Pm[i][j] += F[i][k] * Sm[k][j];
            }
        }
}

static void stress_nh(const double H[3][3], double lam, double mu, double P[3][3]) {
    double Pk[3][3], Pm[3][3], kappa = lam + 2.0 * mu / 3.0;
    nh_parts(H, Pk, Pm);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) P[i][j] = kappa * Pk[i][j] + mu * Pm[i][j];
}

/* A.3 energy: 1/4 kappa (det C - log det C - 1) + 1/2 mu ((det C)^(-1/3) tr C - 3) */
static double energy_nh(const double H[3][3], double lam, double mu) {
    double F[3][3], C[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) F[i][j] = H[i][j] + (i == j ? 1.0 : 0.0);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            C[i][j] = 0.0;
            for (int k = 0; k < 3; ++k) C[i][j] += F[k][i] * F[k][j];
        }
    double dC = det3(C), trC = C[0][0] + C[1][1] + C[2][2];
    double kappa = lam + 2.0 * mu / 3.0;
    return 0.25 * kappa * (dC - log(dC) - 1.0) + 0.5 * mu * (pow(dC, -1.0 / 3.0) * trC - 3.0);
}

/* directional derivative dP = (dP/dF)[G] of the NH stress, split as kappa*dPk + mu*dPm.
 * Derived from P = F S(C):  dP = G S + F dS,  dC = G^T F + F^T G,
 * d(det C) = det C tr(C^-1 dC),  d(C^-1) = -C^-1 dC C^-1,  d((det C)^(-1/3)) = -1/3 (det C)^(-1/3) tr(C^-1 dC). */
static void nh_tangent(const double H[3][3], const double G[3][3], double dPk[3][3], double dPm[3][3]) {
    double F[3][3], C[3][3], Ci[3][3], dC[3][3], dCi[3][3], tmp[3][3];
    double Sk[3][3], Sm[3][3], dSk[3][3], dSm[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) F[i][j] = H[i][j] + (i == j ? 1.0 : 0.0);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            C[i][j] = 0.0; dC[i][j] = 0.0;
            for (int k = 0; k < 3; ++k) {
                C[i][j] += F[k][i] * F[k][j];
                dC[i][j] += G[k][i] * F[k][j] + F[k][i] * G[k][j];
            }
        }
    double detC = det3(C);
    inv3(C, Ci);
    double trC = C[0][0] + C[1][1] + C[2][2], dtrC = dC[0][0] + dC[1][1] + dC[2][2];
    double tCidC = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) tCidC += Ci[i][j] * dC[j][i];
    double ddetC = detC * tCidC;
    double g = pow(detC, -1.0 / 3.0), dg = -g * tCidC / 3.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            tmp[i][j] = 0.0;
            for (int k = 0; k < 3; ++k) tmp[i][j] += Ci[i][k] * dC[k][j];
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            dCi[i][j] = 0.0;
            for (int k = 0; k < 3; ++k) dCi[i][j] -= tmp[i][k] * Ci[k][j];
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double d = (i == j ? 1.0 : 0.0);
            Sk[i][j] = 0.5 * (detC - 1.0) * Ci[i][j];
            Sm[i][j] = g * (d - trC * Ci[i][j] / 3.0);
            dSk[i][j] = 0.5 * ddetC * Ci[i][j] + 0.5 * (detC - 1.0) * dCi[i][j];
            dSm[i][j] = dg * (d - trC * Ci[i][j] / 3.0) + g * (-(dtrC * Ci[i][j] + trC * dCi[i][j]) / 3.0);
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            dPk[i][j] = 0.0; dPm[i][j] = 0.0;
            for (int k = 0; k < 3; ++k) {
                dPk[i][j] += G[i][k] * Sk[k][j] + F[i][k] * dSk[k][j];
                dPm[i][j] += G[i][k] * Sm[k][j] + F[i][k] * dSm[k][j];
            }
        }
}

/* A.2 Saint Venant-Kirchhoff: F = I + H, E = 1/2 (F^T F - I) (the printed "1/2 F^T F - I" read as the
 * Green-Lagrange strain), S = lambda tr(E) I + 2 mu E, P = F S. */
static void svk_strain(const double H[3][3], double F[3][3], double E[3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) F[i][j] = H[i][j] + (i == j ? 1.0 : 0.0);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double c = 0.0;
            for (int k = 0; k < 3; ++k) c += F[k][i] * F[k][j];
            E[i][j] = 0.5 * (c - (i == j ? 1.0 : 0.0));
        }
}

static void stress_svk(const double H[3][3], double lam, double mu, double P[3][3]) {
    double F[3][3], E[3][3], S[3][3];
    svk_strain(H, F, E);
    double tr = E[0][0] + E[1][1] + E[2][2];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) S[i][j] = 2.0 * mu * E[i][j] + (i == j ? lam * tr : 0.0);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            P[i][j] = 0.0;
            for (int k = 0; k < 3; ++k) P[i][j] += F[i][k] * S[k][j];
        }
}

/* A.2 energy: lambda/2 (tr E)^2 + mu tr(E^2) */
static double energy_svk(const double H[3][3], double lam, double mu) {
    double F[3][3], E[3][3];
    svk_strain(H, F, E);
    double tr = E[0][0] + E[1][1] + E[2][2], tr2 = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) tr2 += E[i][j] * E[j][i];
    return 0.5 * lam * tr * tr + mu * tr2;
}

/* dP = G S + F dS, dS = lambda tr(dE) I + 2 mu dE, dE = 1/2 (G^T F + F^T G) */
static void svk_tangent(const double H[3][3], const double G[3][3], double lam, double mu, double dP[3][3]) {
    double F[3][3], E[3][3], S[3][3], dE[3][3], dS[3][3];
    svk_strain(H, F, E);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double c = 0.0;
            for (int k = 0; k < 3; ++k) c += G[k][i] * F[k][j] + F[k][i] * G[k][j];
            dE[i][j] = 0.5 * c;
        }
    double tr = E[0][0] + E[1][1] + E[2][2], dtr = dE[0][0] + dE[1][1] + dE[2][2];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            S[i][j] = 2.0 * mu * E[i][j] + (i == j ? lam * tr : 0.0);
            dS[i][j] = 2.0 * mu * dE[i][j] + (i == j ? lam * dtr : 0.0);
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            dP[i][j] = 0.0;
            for (int k = 0; k < 3; ++k) dP[i][j] += G[i][k] * S[k][j] + F[i][k] * dS[k][j];
        }
}

static void stress(int model, const double H[3][3], double lam, double mu, double P[3][3]) {
    if (model == ORC_NH) stress_nh(H, lam, mu, P);
    else if (model == ORC_SVK) stress_svk(H, lam, mu, P);
    else stress_le(H, lam, mu, P);
}

static double energy(int model, const double H[3][3], double lam, double mu) {
    if (model == ORC_NH) return energy_nh(H, lam, mu);
    if (model == ORC_SVK) return energy_svk(H, lam, mu);
    return energy_le(H, lam, mu);
}

/* ------------------------------------------------------------------------------------------ */
/* element loops                                                                               */
/* ------------------------------------------------------------------------------------------ */
static void gather_elem(const omesh* m, int e, const double* u, int nodes[8], double X[8][3], double U[8][3]) {
    elem_nodes(m, e, nodes);
    for (int a = 0; a < 8; ++a) {
        node_X(m, nodes[a], X[a]);
        for (int c = 0; c < 3; ++c) U[a][c] = u[3 * nodes[a] + c];
    }
}

static void grad_at(const double U[8][3], const double dNdX[8][3], double H[3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            H[i][j] = 0.0;
            for (int a = 0; a < 8; ++a) H[i][j] += U[a][i] * dNdX[a][j];
        }
}

/* f_int (interleaved, length 3*nn) = sum over elements and Gauss points of w detJ P grad N */
static void internal_force(const omesh* m, int model, double lam, double mu, const double* lam_e,
                           const double* mu_e, const double* u, double* f) {
    memset(f, 0, sizeof(double) * 3 * (size_t)m->nn);
    for (int e = 0; e < m->ne; ++e) {
        int nodes[8];
        double X[8][3], U[8][3], dNdX[8][3], H[3][3], P[3][3];
        double le = lam_e ? lam_e[e] : lam, me = mu_e ? mu_e[e] : mu;
        gather_elem(m, e, u, nodes, X, U);
        for (int g = 0; g < 8; ++g) {
            double detJ = physical_gradients(X, g, dNdX);
            grad_at(U, dNdX, H);
            stress(model, H, le, me, P);
            for (int a = 0; a < 8; ++a)
                for (int i = 0; i < 3; ++i) {
                    double s = 0.0;
                    for (int j = 0; j < 3; ++j) s += P[i][j] * dNdX[a][j];
                    f[3 * nodes[a] + i] += detJ * s; /* Gauss weight 1 */
                }
        }
    }
}

static void lumped_mass(const omesh* m, double rho, double* mass) {
    memset(mass, 0, sizeof(double) * (size_t)m->nn);
    for (int e = 0; e < m->ne; ++e) {
        int nodes[8];
        double X[8][3], dNdX[8][3], V = 0.0;
        elem_nodes(m, e, nodes);
        for (int a = 0; a < 8; ++a) node_X(m, nodes[a], X[a]);
        for (int g = 0; g < 8; ++g) V += physical_gradients(X, g, dNdX);
        for (int a = 0; a < 8; ++a) mass[nodes[a]] += rho * V / 8.0;
    }
}

/* ------------------------------------------------------------------------------------------ */
/* stability limit of the explicit scheme                                                      */
/* ------------------------------------------------------------------------------------------ */
/* Central differences (Newmark beta = 0, gamma = 1/2) are stable for omega_max dt <= 2, where
 * omega_max^2 is the largest eigenvalue of M^-1 K, K the stiffness at the reference configuration
 * (linear elastic with (lambda, mu); the Neo-Hookean law of Appendix A linearises to the same).  With
 * a lumped mass, omega_max^2 never exceeds the largest eigenvalue of any element's own M_e^-1 K_e
 * (the element eigenvalue inequality of Irons and Treharne), so the oracle takes that bound: it forms
 * K_e column by column from the linear elastic force of unit nodal displacements, M_e = rho V_e / 8
 * per node, and finds the largest eigenvalue by the cyclic Jacobi method. */
static void element_stiffness(const double X[8][3], double lam, double mu, double K[24][24]) {
    for (int col = 0; col < 24; ++col) {
        double U[8][3] = {{0}};
        U[col / 3][col % 3] = 1.0;
        double f[24] = {0};
        for (int g = 0; g < 8; ++g) {
            double dNdX[8][3], H[3][3], P[3][3];
            double detJ = physical_gradients(X, g, dNdX);
            grad_at(U, dNdX, H);
            stress_le(H, lam, mu, P);
            for (int a = 0; a < 8; ++a)
                for (int i = 0; i < 3; ++i) {
                    double t = 0.0;
                    for (int j = 0; j < 3; ++j) t += P[i][j] * dNdX[a][j];
                    f[3 * a + i] += detJ * t;
                }
        }
        for (int row = 0; row < 24; ++row) K[row][col] = f[row];
    }
}

/* largest eigenvalue of a symmetric n x n matrix (row-major, overwritten) by cyclic Jacobi rotations */
static double jacobi_max_eig(double* A, int n) {
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int i = 0; i < n; ++i) {
            diag += A[i * n + i] * A[i * n + i];
            for (int j = i + 1; j < n; ++j) off += A[i * n + j] * A[i * n + j];
        }
        if (off <= 1e-30 * diag) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[p * n + q];
                if (apq == 0.0) continue;
                double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < n; ++k) { /* columns p, q */
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - sn * akq;
                    A[k * n + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) { /* rows p, q */
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - sn * aqk;
                    A[q * n + k] = sn * apk + c * aqk;
                }
            }
    }
    double m = A[0];
    for (int i = 1; i < n; ++i) m = fmax(m, A[i * n + i]);
    return m;
}

/* max over elements of the largest eigenvalue of M_e^-1 K_e.  The eigenproblem is solved again only
 * when an element's material differs from the previous element's or its volume differs by more than
 * rounding (1e-12 relative): on a box of equal cubes the element matrices differ only in the last bits
 * of their node coordinates. */
static double max_element_omega2(const omesh* m, double lam, double mu, const double* lam_e, const double* mu_e,
                                 double rho) {
    double best = 0.0, last_l = NAN, last_m = NAN, last_v = NAN, last_w = 0.0;
    for (int e = 0; e < m->ne; ++e) {
        int nodes[8];
        double X[8][3], dNdX[8][3], V = 0.0;
        elem_nodes(m, e, nodes);
        for (int a = 0; a < 8; ++a) node_X(m, nodes[a], X[a]);
        for (int g = 0; g < 8; ++g) V += physical_gradients(X, g, dNdX);
        double le = lam_e ? lam_e[e] : lam, me = mu_e ? mu_e[e] : mu;
        double w;
        if (le == last_l && me == last_m && fabs(V - last_v) <= 1e-12 * fabs(last_v)) {
            w = last_w;
        } else {
            double K[24][24], A[24 * 24];
            element_stiffness(X, le, me, K);
            for (int i = 0; i < 24; ++i)
                for (int j = 0; j < 24; ++j) A[i * 24 + j] = 0.5 * (K[i][j] + K[j][i]) * 8.0 / (rho * V);
            w = jacobi_max_eig(A, 24);
            last_l = le; last_m = me; last_v = V; last_w = w;
        }
        if (!(w == w)) return w; /* NaN propagates */
        best = fmax(best, w);
    }
    return best;
}

/* largest stable explicit time step 2 / omega_max by the element bound; 0 for a material whose
 * reference stiffness is not positive definite on the deformation modes (mu <= 0 or 3 lambda + 2 mu <= 0) */
double orc_stable_dt(int nx, int ny, int nz, double h, const double* org, double lam, double mu,
                     const double* lam_e, const double* mu_e, double rho) {
    omesh m;
    mesh_set(&m, nx, ny, nz, h, org);
    for (int e = 0; e < m.ne; ++e) {
        double le = lam_e ? lam_e[e] : lam, me = mu_e ? mu_e[e] : mu;
        if (!(me > 0.0) || !(3.0 * le + 2.0 * me > 0.0)) return 0.0;
    }
    if (!(rho > 0.0)) return 0.0;
    double w = max_element_omega2(&m, lam, mu, lam_e, mu_e, rho);
    if (!(w > 0.0)) return 0.0;
    return 2.0 / sqrt(w);
}

/* ------------------------------------------------------------------------------------------ */
/* exported element-level entry points (used by the pin tests)                                 */
/* ------------------------------------------------------------------------------------------ */
int orc_internal_force(int nx, int ny, int nz, double h, const double* org, int model, double lam, double mu,
                       const double* lam_e, const double* mu_e, const double* u, double* f) {
    omesh m;
    mesh_set(&m, nx, ny, nz, h, org);
    internal_force(&m, model, lam, mu, lam_e, mu_e, u, f);
    return ORC_OK;
}

double orc_strain_energy(int nx, int ny, int nz, double h, const double* org, int model, double lam, double mu,
                         const double* lam_e, const double* mu_e, const double* u) {
    omesh m;
    mesh_set(&m, nx, ny, nz, h, org);
    double E = 0.0;
    for (int e = 0; e < m.ne; ++e) {
        int nodes[8];
        double X[8][3], U[8][3], dNdX[8][3], H[3][3];
        double le = lam_e ? lam_e[e] : lam, me = mu_e ? mu_e[e] : mu;
        gather_elem(&m, e, u, nodes, X, U);
        for (int g = 0; g < 8; ++g) {
            double detJ = physical_gradients(X, g, dNdX);
            grad_at(U, dNdX, H);
            E += detJ * energy(model, H, le, me);
        }
    }
    return E;
}

int orc_stress(int model, const double* H, double lam, double mu, double* P) {
    double Hm[3][3], Pm[3][3];
    for (int i = 0; i < 9; ++i) Hm[i / 3][i % 3] = H[i];
    stress(model, Hm, lam, mu, Pm);
    for (int i = 0; i < 9; ++i) P[i] = Pm[i / 3][i % 3];
    return ORC_OK;
}

double orc_energy_density(int model, const double* H, double lam, double mu) {
    double Hm[3][3];
    for (int i = 0; i < 9; ++i) Hm[i / 3][i % 3] = H[i];
    return energy(model, Hm, lam, mu);
}

void orc_lumped_mass(int nx, int ny, int nz, double h, const double* org, double rho, double* mass) {
    omesh m;
    mesh_set(&m, nx, ny, nz, h, org);
    lumped_mass(&m, rho, mass);
}

/* Vector-Jacobian product of the internal force: given ybar (3*nn),
 *   ubar = (df/du)^T ybar,  lam_bar[e] = ybar . df/dlam_e,  mu_bar[e] = ybar . df/dmu_e.
 * The tangent of a hyperelastic law has major symmetry, so (dP/dF)^T[G] = (dP/dF)[G]. */
static void force_vjp(const omesh* m, int model, const double* lam_e, const double* mu_e, const double* u,
                      const double* ybar, double* ubar, double* lam_bar, double* mu_bar) {
    memset(ubar, 0, sizeof(double) * 3 * (size_t)m->nn);
    for (int e = 0; e < m->ne; ++e) {
        int nodes[8];
        double X[8][3], U[8][3], Y[8][3], dNdX[8][3], H[3][3], G[3][3];
        double le = lam_e[e], me = mu_e[e], lb = 0.0, mb = 0.0;
        gather_elem(m, e, u, nodes, X, U);
        for (int a = 0; a < 8; ++a)
            for (int c = 0; c < 3; ++c) Y[a][c] = ybar[3 * nodes[a] + c];
        for (int g = 0; g < 8; ++g) {
            double detJ = physical_gradients(X, g, dNdX), dP[3][3];
            grad_at(U, dNdX, H);
            grad_at(Y, dNdX, G);
            if (model == ORC_NH) {
                double dPk[3][3], dPm[3][3], Pk[3][3], Pm[3][3], kappa = le + 2.0 * me / 3.0;
                nh_tangent(H, G, dPk, dPm);
                nh_parts(H, Pk, Pm);
                double sk = 0.0, sm = 0.0;
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) {
                        dP[i][j] = kappa * dPk[i][j] + me * dPm[i][j];
                        sk += Pk[i][j] * G[i][j];
                        sm += Pm[i][j] * G[i][j];
                    }
                /* d kappa / d lambda = 1, d kappa / d mu = 2/3 */
                lb += detJ * sk;
                mb += detJ * (sm + 2.0 * sk / 3.0);
            } else {
                stress_le(G, le, me, dP); /* linear: the tangent applied to G is sigma(G) */
                double epsH[3][3], trH = H[0][0] + H[1][1] + H[2][2], sl = 0.0, sm = 0.0;
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) epsH[i][j] = 0.5 * (H[i][j] + H[j][i]);
                for (int i = 0; i < 3; ++i) {
                    sl += trH * G[i][i];
                    for (int j = 0; j < 3; ++j) sm += 2.0 * epsH[i][j] * G[i][j];
                }
                lb += detJ * sl;
                mb += detJ * sm;
            }
            for (int a = 0; a < 8; ++a)
                for (int i = 0; i < 3; ++i) {
                    double s = 0.0;
                    for (int j = 0; j < 3; ++j) s += dP[i][j] * dNdX[a][j];
                    ubar[3 * nodes[a] + i] += detJ * s;
                }
        }
        if (lam_bar) lam_bar[e] = lb;
        if (mu_bar) mu_bar[e] = mb;
    }
}

int orc_force_vjp(int nx, int ny, int nz, double h, const double* org, int model, const double* lam_e,
                  const double* mu_e, const double* u, const double* ybar, double* ubar, double* lam_bar,
                  double* mu_bar) {
    if (model == ORC_SVK) return ORC_EINVAL; /* the adjoint covers LE and NH */
    omesh m;
    mesh_set(&m, nx, ny, nz, h, org);
    force_vjp(&m, model, lam_e, mu_e, u, ybar, ubar, lam_bar, mu_bar);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* spatial projector Pi: donor element search and trilinear weights                            */
/* ------------------------------------------------------------------------------------------ */
#define XI_TOL 1e-9

/* invert the trilinear map of element e at point x by Newton; returns 1 if the point lies in the
 * element (all |xi| <= 1 + XI_TOL), with xi snapped to +-1 within XI_TOL */
static int locate_in_element(const omesh* m, int e, const double x[3], double xi[3]) {
    int nodes[8];
    double X[8][3];
    elem_nodes(m, e, nodes);
    for (int a = 0; a < 8; ++a) node_X(m, nodes[a], X[a]);
    xi[0] = xi[1] = xi[2] = 0.0;
    for (int it = 0; it < 30; ++it) {
        double N[8], dN[8][3], r[3] = {0, 0, 0}, J[3][3] = {{0}}, Ji[3][3];
        shape(xi, N, dN);
        for (int a = 0; a < 8; ++a)
            for (int i = 0; i < 3; ++i) {
                r[i] += N[a] * X[a][i];
                for (int j = 0; j < 3; ++j) J[i][j] += X[a][i] * dN[a][j];
            }
        for (int i = 0; i < 3; ++i) r[i] -= x[i];
        inv3(J, Ji);
        double step = 0.0;
        for (int i = 0; i < 3; ++i) {
            double d = 0.0;
            for (int j = 0; j < 3; ++j) d += Ji[i][j] * r[j];
            xi[i] -= d;
            step += fabs(d);
        }
        if (step < 1e-15) break;
    }
    for (int i = 0; i < 3; ++i) {
        if (fabs(xi[i]) > 1.0 + XI_TOL) return 0;
        if (fabs(xi[i] - 1.0) <= XI_TOL) xi[i] = 1.0;
        if (fabs(xi[i] + 1.0) <= XI_TOL) xi[i] = -1.0;
    }
    return 1;
}

/* per-axis index range of the elements whose extent [org + i h, org + (i+1) h], widened by the
 * containment tolerance, holds coordinate xc; returns 0 if there is none */
static int axis_range(double xc, double org, double h, int n, int* first, int* last) {
    *first = -1; *last = -2;
    for (int i = 0; i < n; ++i) {
        double lo = org + i * h, hi = org + (i + 1) * h, tol = 1e-6 * (hi - lo);
        if (xc < lo - tol || xc > hi + tol) continue;
        if (*first < 0) *first = i;
        *last = i;
    }
    return *first >= 0;
}

/* donor = lowest-index element containing x; weights = N_b(xi).  The mesh is an axis-aligned box of
 * cubes, so an element's node bounding box is the product of its per-axis extents and the elements
 * whose (widened) box holds x are the product of the per-axis index ranges; they are visited in
 * increasing element index (k outer, then j, then i) and each is tested by the Newton inversion. */
static int find_donor(const omesh* m, const double x[3], int nodes[8], double w[8]) {
    int i0, i1, j0, j1, k0, k1;
    if (!axis_range(x[0], m->org[0], m->h, m->nx, &i0, &i1) || !axis_range(x[1], m->org[1], m->h, m->ny, &j0, &j1) ||
        !axis_range(x[2], m->org[2], m->h, m->nz, &k0, &k1))
        return 0;
    for (int k = k0; k <= k1; ++k)
        for (int j = j0; j <= j1; ++j)
            for (int i = i0; i <= i1; ++i) {
                int e = i + m->nx * (j + m->ny * k);
                double xi[3], N[8], dN[8][3];
                if (locate_in_element(m, e, x, xi)) {
                    elem_nodes(m, e, nodes);
                    shape(xi, N, dN);
                    for (int bb = 0; bb < 8; ++bb) w[bb] = N[bb];
                    return 1;
                }
            }
    return 0;
}

int orc_donor(int nx, int ny, int nz, double h, const double* org, const double* x, int* nodes, double* w) {
    omesh m;
    mesh_set(&m, nx, ny, nz, h, org);
    return find_donor(&m, x, nodes, w) ? ORC_OK : ORC_EDONOR;
}

/* ------------------------------------------------------------------------------------------ */
/* coupled problem                                                                             */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int kind;
    omesh m;
    int model;
    double lam, mu, rho;
    double *lam_e, *mu_e;
    unsigned char* dmask; /* per node, bit c set => component c clamped to zero */
    int* srow;            /* per node, Schwarz row or -1 */
    int ns;               /* Schwarz nodes */
    int* snode;           /* row -> node */
    double* mass;
    double *u, *v, *a;    /* [nn][3] */
    double *su, *sv, *sa; /* saved at the controller-step start */
    double *pu, *pv;      /* previous iterate at t_k */
    double* hist;         /* input boundary history [(nsub+1)][3 fields][ns][3] */
    /* ROM */
    int r, rs, nfree;
    int* free_dof;        /* free dof ids (3*node + c) in increasing order */
    int* sdof;            /* Schwarz dof ids in increasing order (3 per Schwarz node) */
    double *Phi, *PhiS, *K, *Hq, *B, *c;
    double *q, *qd, *qdd, *sq, *sqd, *sqdd, *pq, *pqd;
    double* qrec;         /* recorded reduced history [(nsub+1)][3][r] */
    double* Cq;           /* cubic operator [r][r(r+1)(r+2)/6] (COpInf) or NULL */
    double* ghat;
    int rs_rows;          /* declared row count of PhiS */
    /* time integrator of a FOM: 0 explicit central differences, 1 implicit average acceleration */
    int implicit;
    /* substeps per controller interval and their length (Sec. 4.1: Delta t_i = (t_k - t_{k-1}) / n_i) */
    int nsub;
    double dt;
} osub;

typedef struct {
    int dst, src;
    int nrow;
    int* row;    /* Schwarz row of dst */
    int* dnode;  /* [nrow][8] donor nodes in src */
    double* dw;  /* [nrow][8] weights */
    double* rec; /* src trace Pi(u, v, a) at the src's time levels [(nsub_src+1)][3 fields][nrow][3] */
} ocpl;

typedef struct {
    double dt;
    int nsub, max_it;
    double tol_abs, tol_rel;
    int nsd, ncpl;
    osub sd[ORC_MAX_SUB];
    ocpl cpl[ORC_MAX_CPL];
    int initialised;
    /* Schwarz variant: 0 multiplicative (each subdomain uses the data its predecessors published in
     * the same iteration), 1 additive (every subdomain uses the previous iteration's data; Remark
     * additive_sam) */
    int additive;
} oprob;

static void* xcalloc(size_t n, size_t s) { return calloc(n ? n : 1, s); }

void* orc_problem_new(double dt, int nsub, double tol_abs, double tol_rel, int max_it) {
    oprob* p = (oprob*)xcalloc(1, sizeof(oprob));
    p->dt = dt; p->nsub = nsub; p->tol_abs = tol_abs; p->tol_rel = tol_rel; p->max_it = max_it;
    return p;
}

static void sub_free(osub* s) {
    void* ptrs[] = {s->lam_e, s->mu_e, s->dmask, s->srow, s->snode, s->mass, s->u, s->v, s->a, s->su, s->sv,
                    s->sa, s->pu, s->pv, s->hist, s->free_dof, s->sdof, s->Phi, s->PhiS, s->K, s->Hq, s->B,
                    s->c, s->q, s->qd, s->qdd, s->sq, s->sqd, s->sqdd, s->pq, s->pqd, s->qrec, s->ghat, s->Cq};
    for (size_t i = 0; i < sizeof(ptrs) / sizeof(ptrs[0]); ++i) free(ptrs[i]);
}

void orc_problem_free(void* vp) {
    oprob* p = (oprob*)vp;
    if (!p) return;
    for (int i = 0; i < p->nsd; ++i) sub_free(&p->sd[i]);
    for (int i = 0; i < p->ncpl; ++i) {
        free(p->cpl[i].row); free(p->cpl[i].dnode); free(p->cpl[i].dw); free(p->cpl[i].rec);
    }
    free(p);
}

static double* dup_or_zero(const double* src, size_t n) {
    double* d = (double*)xcalloc(n, sizeof(double));
    if (src) memcpy(d, src, n * sizeof(double));
    return d;
}

static osub* add_common(oprob* p, int kind, int nx, int ny, int nz, double h, const double* org,
                        const unsigned char* dmask, const double* u0, const double* v0) {
    if (p->nsd >= ORC_MAX_SUB) return NULL;
    osub* s = &p->sd[p->nsd++];
    memset(s, 0, sizeof(*s));
    s->kind = kind;
    s->nsub = p->nsub;
    s->dt = p->dt;
    mesh_set(&s->m, nx, ny, nz, h, org);
    size_t nn = (size_t)s->m.nn;
    s->dmask = (unsigned char*)xcalloc(nn, 1);
    if (dmask) memcpy(s->dmask, dmask, nn);
    s->srow = (int*)malloc(sizeof(int) * nn);
    for (size_t n = 0; n < nn; ++n) s->srow[n] = -1;
    s->u = dup_or_zero(u0, 3 * nn);
    s->v = dup_or_zero(v0, 3 * nn);
    s->a = dup_or_zero(NULL, 3 * nn);
    s->su = dup_or_zero(NULL, 3 * nn); s->sv = dup_or_zero(NULL, 3 * nn); s->sa = dup_or_zero(NULL, 3 * nn);
    s->pu = dup_or_zero(NULL, 3 * nn); s->pv = dup_or_zero(NULL, 3 * nn);
    /* clamped components start (and stay) at zero */
    for (size_t n = 0; n < nn; ++n)
        for (int c = 0; c < 3; ++c)
            if (s->dmask[n] & (1 << c)) { s->u[3 * n + c] = 0.0; s->v[3 * n + c] = 0.0; }
    return s;
}

int orc_add_fom(void* vp, int nx, int ny, int nz, double h, const double* org, int model, double lam, double mu,
                double rho, const double* lam_e, const double* mu_e, const unsigned char* dmask, const double* u0,
                const double* v0) {
    if (model != ORC_LE && model != ORC_NH && model != ORC_SVK) return ORC_EINVAL;
    oprob* p = (oprob*)vp;
    osub* s = add_common(p, ORC_FOM, nx, ny, nz, h, org, dmask, u0, v0);
    if (!s) return ORC_EINVAL;
    s->model = model; s->lam = lam; s->mu = mu; s->rho = rho;
    if (lam_e) s->lam_e = dup_or_zero(lam_e, (size_t)s->m.ne);
    if (mu_e) s->mu_e = dup_or_zero(mu_e, (size_t)s->m.ne);
    s->mass = (double*)xcalloc((size_t)s->m.nn, sizeof(double));
    lumped_mass(&s->m, rho, s->mass);
    return p->nsd - 1;
}

/* Phi: [nfree][r] row-major over the ROM subdomain's free dofs; PhiS: [3*ns][rs] over its Schwarz
 * dofs; K [r][r]; H [r][r(r+1)/2]; B [r][rs]; c [r]. */
int orc_add_rom(void* vp, int nx, int ny, int nz, double h, const double* org, const unsigned char* dmask, int r,
                int rs, int nfree, int nsdof, const double* Phi, const double* PhiS, const double* K, const double* H,
                const double* B, const double* c, const double* u0, const double* v0) {
    oprob* p = (oprob*)vp;
    osub* s = add_common(p, ORC_ROM, nx, ny, nz, h, org, dmask, u0, v0);
    if (!s) return ORC_EINVAL;
    s->r = r; s->rs = rs;
    /* row counts are checked against the coupling masks in orc_init */
    s->nfree = nfree;
    s->Phi = dup_or_zero(Phi, (size_t)nfree * r);
    s->PhiS = dup_or_zero(PhiS, (size_t)nsdof * rs);
    s->rs_rows = nsdof;
    size_t nq = (size_t)r * (r + 1) / 2;
    s->K = dup_or_zero(K, (size_t)r * r);
    s->Hq = dup_or_zero(H, (size_t)r * nq);
    s->B = dup_or_zero(B, (size_t)r * rs);
    s->c = dup_or_zero(c, (size_t)r);
    s->q = dup_or_zero(NULL, r); s->qd = dup_or_zero(NULL, r); s->qdd = dup_or_zero(NULL, r);
    s->sq = dup_or_zero(NULL, r); s->sqd = dup_or_zero(NULL, r); s->sqdd = dup_or_zero(NULL, r);
    s->pq = dup_or_zero(NULL, r); s->pqd = dup_or_zero(NULL, r);
    s->ghat = dup_or_zero(NULL, rs);
    return p->nsd - 1;
}

int orc_couple(void* vp, int dst, int src, const unsigned char* nodes) {
    oprob* p = (oprob*)vp;
    if (p->ncpl >= ORC_MAX_CPL || dst < 0 || src < 0 || dst >= p->nsd || src >= p->nsd || dst == src)
        return ORC_EINVAL;
    osub* d = &p->sd[dst];
    ocpl* cp = &p->cpl[p->ncpl++];
    memset(cp, 0, sizeof(*cp));
    cp->dst = dst; cp->src = src;
    /* rows are assigned after all couplings are known (increasing node order); store the mask now */
    cp->row = (int*)xcalloc((size_t)d->m.nn, sizeof(int));
    for (int n = 0; n < d->m.nn; ++n) cp->row[n] = nodes[n] ? 1 : 0;
    return p->ncpl - 1;
}

static int is_free(const osub* s, int n, int c) { return !(s->dmask[n] & (1 << c)) && s->srow[n] < 0; }

/* full-field value (fields 0,1,2 = u,v,a) of a subdomain at node n, component c.
 * ROM: free dofs are Phi q (or qd, qdd); clamped dofs are 0; Schwarz dofs carry the ROM's current
 * boundary data (history slot `slot`). */
static double rom_field(const oprob* p, const osub* s, int field, int n, int c, const double* qv, int slot) {
    if (s->dmask[n] & (1 << c)) return 0.0;
    if (s->srow[n] >= 0) {
        size_t ns = (size_t)s->ns;
        return s->hist[((size_t)slot * 3 + field) * ns * 3 + (size_t)s->srow[n] * 3 + c];
    }
    int dof = 3 * n + c;
    /* binary search of dof in free_dof */
    int lo = 0, hi = s->nfree - 1, row = -1;
    while (lo <= hi) {
        int mid = (lo + hi) / 2;
        if (s->free_dof[mid] == dof) { row = mid; break; }
        if (s->free_dof[mid] < dof) lo = mid + 1; else hi = mid - 1;
    }
    (void)p;
    double val = 0.0;
    for (int k = 0; k < s->r; ++k) val += s->Phi[(size_t)row * s->r + k] * qv[k];
    return val;
}

/* record Pi(src fields) at the src's time level `level` into the coupling's trace (Sec. 4.1, the
 * pointwise spatial projector).  FOM src: from its current (u, v, a).  ROM src: from its recorded
 * reduced history at `level`, or from its current (q, qd, qdd) when zoh is set. */
static void trace_level(oprob* p, const ocpl* cp, int level, int zoh) {
    const osub* s = &p->sd[cp->src];
    size_t nr = (size_t)cp->nrow;
    for (int i = 0; i < cp->nrow; ++i) {
        for (int f = 0; f < 3; ++f)
            for (int c = 0; c < 3; ++c) {
                double val = 0.0;
                for (int b = 0; b < 8; ++b) {
                    int n = cp->dnode[8 * i + b];
                    double w = cp->dw[8 * i + b];
                    double x;
                    if (w == 0.0) continue;
                    if (s->kind == ORC_FOM) {
                        const double* fld = f == 0 ? s->u : (f == 1 ? s->v : s->a);
                        x = fld[3 * n + c];
                    } else {
                        const double* qv;
                        if (zoh) qv = f == 0 ? s->q : (f == 1 ? s->qd : s->qdd);
                        else qv = s->qrec + ((size_t)level * 3 + f) * s->r;
                        x = rom_field(p, s, f, n, c, qv, zoh ? 0 : level);
                    }
                    val += w * x;
                }
                cp->rec[((size_t)level * 3 + f) * nr * 3 + (size_t)i * 3 + c] = val;
            }
    }
}

/* Temporal interpolant Xi (Sec. 4.1, Fig. schwarz_time_discretization): the data of dst level m
 * (time t_{k-1} + m T / n_dst) from the src trace at levels l = 0..n_src (times t_{k-1} + l T / n_src),
 * linear between the two levels that bracket it; an exact level is copied. */
static void publish(oprob* p, const ocpl* cp) {
    osub* d = &p->sd[cp->dst];
    int ns_ = p->sd[cp->src].nsub, nd = d->nsub;
    size_t nr = (size_t)cp->nrow, dns = (size_t)d->ns;
    for (int m = 1; m <= nd; ++m) {
        long long num = (long long)m * ns_;
        int l = (int)(num / nd);
        long long rem = num - (long long)l * nd;
        double w = (double)rem / (double)nd;
        for (int f = 0; f < 3; ++f)
            for (int i = 0; i < cp->nrow; ++i)
                for (int c = 0; c < 3; ++c) {
                    double x0 = cp->rec[((size_t)l * 3 + f) * nr * 3 + (size_t)i * 3 + c];
                    double val = x0;
                    if (rem != 0) {
                        double x1 = cp->rec[((size_t)(l + 1) * 3 + f) * nr * 3 + (size_t)i * 3 + c];
                        val = (1.0 - w) * x0 + w * x1;
                    }
                    d->hist[((size_t)m * 3 + f) * dns * 3 + (size_t)cp->row[i] * 3 + c] = val;
                }
    }
}

/* zero-order hold of the src's current state: trace level 0 and every dst level */
static void zoh(oprob* p, const ocpl* cp) {
    osub* d = &p->sd[cp->dst];
    size_t nr = (size_t)cp->nrow, dns = (size_t)d->ns;
    trace_level(p, cp, 0, 1);
    for (int m = 0; m <= d->nsub; ++m)
        for (int f = 0; f < 3; ++f)
            for (int i = 0; i < cp->nrow; ++i)
                for (int c = 0; c < 3; ++c)
                    d->hist[((size_t)m * 3 + f) * dns * 3 + (size_t)cp->row[i] * 3 + c] =
                        cp->rec[((size_t)f) * nr * 3 + (size_t)i * 3 + c];
}

/* ROM right-hand side: K q + H kron_c(q) [+ C kron3_c(q)] + B ghat + c, kron_c(q) = (q_i q_j)_{i<=j}
 * and kron3_c(q) = (q_i q_j q_k)_{i<=j<=k}, both in lexicographic (row-major) order */
static void rom_rhs(const osub* s, const double* q, const double* ghat, double* out) {
    int r = s->r;
    size_t nq = (size_t)r * (r + 1) / 2, nc = (size_t)r * (r + 1) * (r + 2) / 6;
    for (int i = 0; i < r; ++i) {
        double acc = s->c[i];
        for (int j = 0; j < r; ++j) acc += s->K[(size_t)i * r + j] * q[j];
        size_t col = 0;
        for (int j = 0; j < r; ++j)
            for (int k = j; k < r; ++k) acc += s->Hq[(size_t)i * nq + col++] * q[j] * q[k];
        if (s->Cq) {
            col = 0;
            for (int j = 0; j < r; ++j)
                for (int k = j; k < r; ++k)
                    for (int l = k; l < r; ++l) acc += s->Cq[(size_t)i * nc + col++] * q[j] * q[k] * q[l];
        }
        for (int j = 0; j < s->rs; ++j) acc += s->B[(size_t)i * s->rs + j] * ghat[j];
        out[i] = acc;
    }
}

/* ghat = Phi_S^T s, s = the ROM's Schwarz displacement data at history slot `slot` */
static void rom_ghat(const osub* s, int slot) {
    size_t ns = (size_t)s->ns;
    const double* su = s->hist + (size_t)slot * 3 * ns * 3; /* field 0 */
    for (int k = 0; k < s->rs; ++k) {
        double acc = 0.0;
        for (size_t i = 0; i < 3 * ns; ++i) acc += s->PhiS[i * s->rs + k] * su[i];
        s->ghat[k] = acc;
    }
}

/* time integrator of FOM subdomain i: 0 explicit central differences, 1 implicit average acceleration */
int orc_set_implicit(void* vp, int i, int implicit) {
    oprob* p = (oprob*)vp;
    if (i < 0 || i >= p->nsd || p->sd[i].kind != ORC_FOM) return ORC_EINVAL;
    p->sd[i].implicit = implicit != 0;
    return ORC_OK;
}

/* cubic operator C [r][r(r+1)(r+2)/6] of ROM subdomain i (cubic OpInf; NULL keeps it quadratic) */
int orc_set_rom_cubic(void* vp, int i, const double* C) {
    oprob* p = (oprob*)vp;
    if (i < 0 || i >= p->nsd || p->sd[i].kind != ORC_ROM || p->initialised) return ORC_EINVAL;
    osub* s = &p->sd[i];
    free(s->Cq);
    s->Cq = C ? dup_or_zero(C, (size_t)s->r * ((size_t)s->r * (s->r + 1) * (s->r + 2) / 6)) : NULL;
    return ORC_OK;
}

/* Schwarz variant of the controller: 0 multiplicative, 1 additive */
int orc_set_additive(void* vp, int additive) {
    oprob* p = (oprob*)vp;
    if (p->initialised) return ORC_EINVAL;
    p->additive = additive != 0;
    return ORC_OK;
}

/* substeps of subdomain i per controller interval (its time step is the interval length over n) */
int orc_set_substeps(void* vp, int i, int n) {
    oprob* p = (oprob*)vp;
    if (i < 0 || i >= p->nsd || n < 1 || p->initialised) return ORC_EINVAL;
    p->sd[i].nsub = n;
    p->sd[i].dt = n == p->nsub ? p->dt : (p->dt * (double)p->nsub) / (double)n;
    return ORC_OK;
}

int orc_init(void* vp) {
    oprob* p = (oprob*)vp;
    /* explicit stability: every FOM subdomain's time step within its element bound (a relative
     * allowance of 1e-9 keeps a step exactly at the limit, such as the 1D bar at Courant number 1) */
    for (int i = 0; i < p->nsd; ++i) {
        osub* s = &p->sd[i];
        if (s->kind != ORC_FOM || s->implicit) continue; /* the average-acceleration rule is unconditionally stable */
        double lim = orc_stable_dt(s->m.nx, s->m.ny, s->m.nz, s->m.h, s->m.org, s->lam, s->mu, s->lam_e, s->mu_e,
                                   s->rho);
        if (!(lim > 0.0)) return ORC_EINVAL;
        if (s->dt > lim * (1.0 + 1e-9)) return ORC_ECFL;
    }
    /* Schwarz rows: union of the coupling masks, increasing node order */
    for (int i = 0; i < p->nsd; ++i) {
        osub* s = &p->sd[i];
        int ns = 0;
        for (int n = 0; n < s->m.nn; ++n) {
            int any = 0;
            for (int k = 0; k < p->ncpl; ++k)
                if (p->cpl[k].dst == i && p->cpl[k].row[n]) any = 1;
            if (any) s->srow[n] = ns++;
        }
        s->ns = ns;
        s->snode = (int*)xcalloc((size_t)ns, sizeof(int));
        for (int n = 0; n < s->m.nn; ++n)
            if (s->srow[n] >= 0) s->snode[s->srow[n]] = n;
        s->hist = dup_or_zero(NULL, (size_t)(s->nsub + 1) * 3 * ns * 3);
    }
    /* couplings: donor search */
    for (int k = 0; k < p->ncpl; ++k) {
        ocpl* cp = &p->cpl[k];
        osub* d = &p->sd[cp->dst];
        osub* s = &p->sd[cp->src];
        int* mask = cp->row;
        int cnt = 0;
        for (int n = 0; n < d->m.nn; ++n) cnt += mask[n] ? 1 : 0;
        cp->nrow = cnt;
        int* row = (int*)xcalloc((size_t)cnt, sizeof(int));
        cp->dnode = (int*)xcalloc((size_t)cnt * 8, sizeof(int));
        cp->dw = (double*)xcalloc((size_t)cnt * 8, sizeof(double));
        int t = 0;
        for (int n = 0; n < d->m.nn; ++n) {
            if (!mask[n]) continue;
            double x[3];
            node_X(&d->m, n, x);
            row[t] = d->srow[n];
            if (!find_donor(&s->m, x, cp->dnode + 8 * t, cp->dw + 8 * t)) { free(mask); cp->row = row; return ORC_EDONOR; }
            ++t;
        }
        free(mask);
        cp->row = row;
        cp->rec = dup_or_zero(NULL, (size_t)(s->nsub + 1) * 3 * (size_t)cnt * 3);
    }
    for (int k = 0; k < p->ncpl; ++k) {
        ocpl* cp = &p->cpl[k];
        osub* s = &p->sd[cp->src];
        if (s->kind != ORC_ROM) continue;
        for (int t = 0; t < 8 * cp->nrow; ++t)
            if (cp->dw[t] != 0.0 && s->srow[cp->dnode[t]] >= 0) return ORC_EINVAL;
    }
    /* ROM dof maps and operator copies */
    for (int i = 0; i < p->nsd; ++i) {
        osub* s = &p->sd[i];
        if (s->kind != ORC_ROM) continue;
        int nf = 0;
        for (int n = 0; n < s->m.nn; ++n)
            for (int c = 0; c < 3; ++c) nf += is_free(s, n, c);
        if (nf != s->nfree || 3 * s->ns != s->rs_rows) return ORC_EINVAL;
        s->free_dof = (int*)xcalloc((size_t)nf, sizeof(int));
        int t = 0;
        for (int n = 0; n < s->m.nn; ++n)
            for (int c = 0; c < 3; ++c)
                if (is_free(s, n, c)) s->free_dof[t++] = 3 * n + c;
        s->qrec = dup_or_zero(NULL, (size_t)(s->nsub + 1) * 3 * s->r);
        /* q0 = Phi^T u0, qd0 = Phi^T v0 over the free dofs */
        for (int k = 0; k < s->r; ++k) {
            double a = 0.0, b = 0.0;
            for (int f = 0; f < nf; ++f) {
                a += s->Phi[(size_t)f * s->r + k] * s->u[s->free_dof[f]];
                b += s->Phi[(size_t)f * s->r + k] * s->v[s->free_dof[f]];
            }
            s->q[k] = a; s->qd[k] = b;
        }
    }
    /* initial boundary data: zero-order hold of the sources' initial states in every slot */
    for (int k = 0; k < p->ncpl; ++k) zoh(p, &p->cpl[k]);
    /* initial accelerations */
    for (int i = 0; i < p->nsd; ++i) {
        osub* s = &p->sd[i];
        if (s->kind == ORC_FOM) {
            double* f = (double*)xcalloc(3 * (size_t)s->m.nn, sizeof(double));
            internal_force(&s->m, s->model, s->lam, s->mu, s->lam_e, s->mu_e, s->u, f);
            for (int n = 0; n < s->m.nn; ++n)
                for (int c = 0; c < 3; ++c)
                    s->a[3 * n + c] = (s->dmask[n] & (1 << c)) ? 0.0 : -f[3 * n + c] / s->mass[n];
            free(f);
        } else {
            rom_ghat(s, 0);
            rom_rhs(s, s->q, s->ghat, s->qdd);
        }
    }
    p->initialised = 1;
    return ORC_OK;
}

/* record the reduced state at slot j */
static void rom_record(osub* s, int j) {
    memcpy(s->qrec + ((size_t)j * 3 + 0) * s->r, s->q, sizeof(double) * s->r);
    memcpy(s->qrec + ((size_t)j * 3 + 1) * s->r, s->qd, sizeof(double) * s->r);
    memcpy(s->qrec + ((size_t)j * 3 + 2) * s->r, s->qdd, sizeof(double) * s->r);
}

/* advance subdomain i over the controller interval (nsub substeps) with its input history */
/* ------------------------------------------------------------------------------------------ */
/* implicit Newmark (beta = 1/4, gamma = 1/2: average acceleration), Sec. 4.1 with reading c1     */
/* ------------------------------------------------------------------------------------------ */
/* element tangent K_e(u) (24 x 24, element dof order 3*a + i): column q is the directional
 * derivative of the element force along the unit vector of element dof q (Appendix A tangents) */
static void element_tangent(const omesh* m, int model, double lam, double mu, int e, const double* u,
                            double Ke[24][24], int nodes[8]) {
    double X[8][3], U[8][3], dNdX[8][3], H[3][3], G[3][3], dP[3][3];
    gather_elem(m, e, u, nodes, X, U);
    for (int q = 0; q < 24; ++q)
        for (int r = 0; r < 24; ++r) Ke[r][q] = 0.0;
    for (int g = 0; g < 8; ++g) {
        double detJ = physical_gradients(X, g, dNdX);
        grad_at(U, dNdX, H);
        for (int q = 0; q < 24; ++q) {
            double Y[8][3] = {{0}};
            Y[q / 3][q % 3] = 1.0;
            grad_at(Y, dNdX, G);
            if (model == ORC_NH) {
                double dPk[3][3], dPm[3][3], kappa = lam + 2.0 * mu / 3.0;
                nh_tangent(H, G, dPk, dPm);
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) dP[i][j] = kappa * dPk[i][j] + mu * dPm[i][j];
            } else if (model == ORC_SVK) {
                svk_tangent(H, G, lam, mu, dP);
            } else {
                stress_le(G, lam, mu, dP);
            }
            for (int a = 0; a < 8; ++a)
                for (int i = 0; i < 3; ++i) {
                    double t = 0.0;
                    for (int j = 0; j < 3; ++j) t += dP[i][j] * dNdX[a][j];
                    Ke[3 * a + i][q] += detJ * t;
                }
        }
    }
}

/* tangent action y = K(u) p of the assembled element tangents (test entry point) */
int orc_tangent_action(int nx, int ny, int nz, double h, const double* org, int model, double lam, double mu,
                       const double* u, const double* p, double* y) {
    omesh m;
    mesh_set(&m, nx, ny, nz, h, org);
    memset(y, 0, sizeof(double) * 3 * (size_t)m.nn);
    for (int e = 0; e < m.ne; ++e) {
        double Ke[24][24];
        int nodes[8];
        element_tangent(&m, model, lam, mu, e, u, Ke, nodes);
        for (int r = 0; r < 24; ++r) {
            double acc = 0.0;
            for (int q = 0; q < 24; ++q) acc += Ke[r][q] * p[3 * nodes[q / 3] + q % 3];
            y[3 * nodes[r / 3] + r % 3] += acc;
        }
    }
    return ORC_OK;
}

/* Cholesky solve of the dense SPD system A x = b (n x n, row-major, overwritten); 0 if not SPD */
static int dense_spd_solve(double* A, int n, double* b) {
    for (int j = 0; j < n; ++j) {
        double d = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
        if (!(d > 0.0)) return 0;
        d = sqrt(d);
        A[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double t = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) t -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
            A[(size_t)i * n + j] = t / d;
        }
    }
    for (int i = 0; i < n; ++i) {
        double t = b[i];
        for (int k = 0; k < i; ++k) t -= A[(size_t)i * n + k] * b[k];
        b[i] = t / A[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double t = b[i];
        for (int k = i + 1; k < n; ++k) t -= A[(size_t)k * n + i] * b[k];
        b[i] = t / A[(size_t)i * n + i];
    }
    return 1;
}

/* One implicit substep of FOM subdomain s with boundary data h1 (history slot of the new level).
 * Predictor ut = u + dt v + (1/2 - beta) dt^2 a on free dofs; solve R(u) = M (u - ut) / (beta dt^2)
 * + f_int(u) = 0 by Newton's method with the exact tangent M / (beta dt^2) + K(u) (assembled densely,
 * Cholesky), until |R| <= 1e-12 |R(ut)| or an increment |du|^2 <= 1e-28 |u|^2 (at most 25 iterations);
 * then a = (u - ut) / (beta dt^2) and v += dt ((1 - gamma) a_old + gamma a).  Returns 0, or -3 for a
 * non-finite or failed solve. */
static int implicit_substep(osub* s, double dt, const double* h1, size_t ns) {
    const double beta = 0.25, gamma = 0.5, c0 = 1.0 / (beta * dt * dt);
    size_t nn = (size_t)s->m.nn;
    int* fid = (int*)xcalloc(3 * nn, sizeof(int)); /* dof -> free index or -1 */
    int nf = 0;
    for (size_t n = 0; n < nn; ++n)
        for (int c = 0; c < 3; ++c) {
            size_t d = 3 * n + c;
            fid[d] = (!(s->dmask[n] & (1 << c)) && s->srow[n] < 0) ? nf++ : -1;
        }
    double* ut = (double*)xcalloc(3 * nn, sizeof(double));
    double* f = (double*)xcalloc(3 * nn, sizeof(double));
    double* R = (double*)xcalloc((size_t)(nf ? nf : 1), sizeof(double));
    double* J = (double*)xcalloc((size_t)(nf ? nf : 1) * (nf ? nf : 1), sizeof(double));
    for (size_t n = 0; n < nn; ++n)
        for (int c = 0; c < 3; ++c) {
            size_t d = 3 * n + c;
            if (s->dmask[n] & (1 << c)) s->u[d] = 0.0;
            else if (s->srow[n] >= 0) s->u[d] = h1[(size_t)s->srow[n] * 3 + c];
            else s->u[d] += dt * s->v[d] + (0.5 - beta) * dt * dt * s->a[d];
            ut[d] = s->u[d];
        }
    int status = -3;
    double r0 = -1.0;
    for (int it = 0; it < 25; ++it) {
        internal_force(&s->m, s->model, s->lam, s->mu, s->lam_e, s->mu_e, s->u, f);
        double rn = 0.0;
        for (size_t d = 0; d < 3 * nn; ++d)
            if (fid[d] >= 0) {
                R[fid[d]] = c0 * s->mass[d / 3] * (s->u[d] - ut[d]) + f[d];
                rn += R[fid[d]] * R[fid[d]];
            }
        rn = sqrt(rn);
        if (!(rn == rn) || isinf(rn)) break;
        if (r0 < 0.0) r0 = rn;
        if (rn <= 1e-12 * r0 || rn == 0.0) { status = 0; break; }
        /* J = M c0 + sum_e K_e on the free dofs */
        memset(J, 0, sizeof(double) * (size_t)nf * nf);
        for (size_t d = 0; d < 3 * nn; ++d)
            if (fid[d] >= 0) J[(size_t)fid[d] * nf + fid[d]] += c0 * s->mass[d / 3];
        for (int e = 0; e < s->m.ne; ++e) {
            double Ke[24][24];
            int nodes[8];
            double le = s->lam_e ? s->lam_e[e] : s->lam, me = s->mu_e ? s->mu_e[e] : s->mu;
            element_tangent(&s->m, s->model, le, me, e, s->u, Ke, nodes);
            for (int r = 0; r < 24; ++r) {
                int fr = fid[3 * nodes[r / 3] + r % 3];
                if (fr < 0) continue;
                for (int q = 0; q < 24; ++q) {
                    int fq = fid[3 * nodes[q / 3] + q % 3];
                    if (fq >= 0) J[(size_t)fr * nf + fq] += Ke[r][q];
                }
            }
        }
        for (int k = 0; k < nf; ++k) R[k] = -R[k];
        if (!dense_spd_solve(J, nf, R)) break;
        double du2 = 0.0, u2 = 0.0;
        for (size_t d = 0; d < 3 * nn; ++d)
            if (fid[d] >= 0) {
                s->u[d] += R[fid[d]];
                du2 += R[fid[d]] * R[fid[d]];
                u2 += s->u[d] * s->u[d];
            }
        /* an increment at the rounding level of u ends the iteration as well (reading: the predictor
         * may already solve the system to rounding, where the relative residual test cannot be met) */
        if (du2 <= 1e-28 * u2) { status = 0; break; }
    }
    if (status == 0) {
        for (size_t n = 0; n < nn; ++n)
            for (int c = 0; c < 3; ++c) {
                size_t d = 3 * n + c;
                if (s->dmask[n] & (1 << c)) { s->v[d] = 0.0; s->a[d] = 0.0; }
                else if (s->srow[n] >= 0) {
                    s->v[d] = h1[ns * 3 + (size_t)s->srow[n] * 3 + c];
                    s->a[d] = h1[2 * ns * 3 + (size_t)s->srow[n] * 3 + c];
                } else {
                    double an = c0 * (s->u[d] - ut[d]);
                    s->v[d] += dt * ((1.0 - gamma) * s->a[d] + gamma * an);
                    s->a[d] = an;
                }
            }
    }
    free(fid); free(ut); free(f); free(R); free(J);
    return status;
}

static void advance(oprob* p, int i) {
    osub* s = &p->sd[i];
    double dt = s->dt;
    size_t ns = (size_t)s->ns;
    if (s->kind == ORC_FOM && s->implicit) {
        for (int j = 0; j < s->nsub; ++j) {
            const double* h1 = s->hist + (size_t)(j + 1) * 3 * ns * 3;
            if (implicit_substep(s, dt, h1, ns) != 0) {
                /* a failed Newton solve leaves a non-finite state for the criterion to report */
                for (size_t d = 0; d < 3 * (size_t)s->m.nn; ++d) s->u[d] = NAN;
            }
            for (int k = 0; k < p->ncpl; ++k)
                if (p->cpl[k].src == i) trace_level(p, &p->cpl[k], j + 1, 0);
        }
    } else if (s->kind == ORC_FOM) {
        size_t nn = (size_t)s->m.nn;
        double* f = (double*)xcalloc(3 * nn, sizeof(double));
        for (int j = 0; j < s->nsub; ++j) {
            const double* h1 = s->hist + (size_t)(j + 1) * 3 * ns * 3;
            /* predictor on free dofs, Dirichlet data on constrained dofs */
            for (size_t n = 0; n < nn; ++n)
                for (int c = 0; c < 3; ++c) {
                    size_t d = 3 * n + c;
                    if (s->dmask[n] & (1 << c)) s->u[d] = 0.0;
                    else if (s->srow[n] >= 0) s->u[d] = h1[(size_t)s->srow[n] * 3 + c];
                    else s->u[d] += dt * s->v[d] + 0.5 * dt * dt * s->a[d];
                }
            internal_force(&s->m, s->model, s->lam, s->mu, s->lam_e, s->mu_e, s->u, f);
            /* corrector */
            for (size_t n = 0; n < nn; ++n)
                for (int c = 0; c < 3; ++c) {
                    size_t d = 3 * n + c;
                    if (s->dmask[n] & (1 << c)) { s->v[d] = 0.0; s->a[d] = 0.0; }
                    else if (s->srow[n] >= 0) {
                        s->v[d] = h1[ns * 3 + (size_t)s->srow[n] * 3 + c];
                        s->a[d] = h1[2 * ns * 3 + (size_t)s->srow[n] * 3 + c];
                    } else {
                        double an = -f[d] / s->mass[n];
                        s->v[d] += 0.5 * dt * (s->a[d] + an);
                        s->a[d] = an;
                    }
                }
            /* record this substep's trace for every subdomain that takes data from this one */
            for (int k = 0; k < p->ncpl; ++k)
                if (p->cpl[k].src == i) trace_level(p, &p->cpl[k], j + 1, 0);
        }
        free(f);
    } else {
        double* qn = (double*)xcalloc((size_t)s->r, sizeof(double));
        rom_record(s, 0);
        for (int j = 0; j < s->nsub; ++j) {
            for (int k = 0; k < s->r; ++k) s->q[k] += dt * s->qd[k] + 0.5 * dt * dt * s->qdd[k];
            rom_ghat(s, j + 1);
            rom_rhs(s, s->q, s->ghat, qn);
            for (int k = 0; k < s->r; ++k) {
                s->qd[k] += 0.5 * dt * (s->qdd[k] + qn[k]);
                s->qdd[k] = qn[k];
            }
            rom_record(s, j + 1);
        }
        free(qn);
        /* ROM -> neighbours: Pi (Phi q) at every recorded level */
        for (int k = 0; k < p->ncpl; ++k)
            if (p->cpl[k].src == i)
                for (int j = 1; j <= s->nsub; ++j) trace_level(p, &p->cpl[k], j, 0);
    }
}

/* the interval's trace of subdomain i, mapped onto each destination's time levels */
static void publish_from(oprob* p, int i) {
    for (int k = 0; k < p->ncpl; ++k)
        if (p->cpl[k].src == i) publish(p, &p->cpl[k]);
}

static void save_state(oprob* p) {
    for (int i = 0; i < p->nsd; ++i) {
        osub* s = &p->sd[i];
        size_t n3 = 3 * (size_t)s->m.nn;
        memcpy(s->su, s->u, n3 * sizeof(double));
        memcpy(s->sv, s->v, n3 * sizeof(double));
        memcpy(s->sa, s->a, n3 * sizeof(double));
        if (s->kind == ORC_ROM) {
            memcpy(s->sq, s->q, sizeof(double) * s->r);
            memcpy(s->sqd, s->qd, sizeof(double) * s->r);
            memcpy(s->sqdd, s->qdd, sizeof(double) * s->r);
        }
    }
}

static void restore_state(oprob* p) {
    for (int i = 0; i < p->nsd; ++i) {
        osub* s = &p->sd[i];
        size_t n3 = 3 * (size_t)s->m.nn;
        memcpy(s->u, s->su, n3 * sizeof(double));
        memcpy(s->v, s->sv, n3 * sizeof(double));
        memcpy(s->a, s->sa, n3 * sizeof(double));
        if (s->kind == ORC_ROM) {
            memcpy(s->q, s->sq, sizeof(double) * s->r);
            memcpy(s->qd, s->sqd, sizeof(double) * s->r);
            memcpy(s->qdd, s->sqdd, sizeof(double) * s->r);
        }
    }
}

/* criterion conv_criterion at t_k: numerator sum_i ||du_i + dt dv_i||^2, denominator
 * sum_i ||u_i + dt v_i||^2 over free dofs (ROM: over q, qd); then remember this iterate */
static void criterion(oprob* p, double* cnum, double* cden, int* nonfinite) {
    double num = 0.0, den = 0.0;
    for (int i = 0; i < p->nsd; ++i) {
        osub* s = &p->sd[i];
        double dt = s->dt;
        if (s->kind == ORC_FOM) {
            for (int n = 0; n < s->m.nn; ++n)
                for (int c = 0; c < 3; ++c) {
                    if (!is_free(s, n, c)) continue;
                    size_t d = 3 * (size_t)n + c;
                    double x = (s->u[d] - s->pu[d]) + dt * (s->v[d] - s->pv[d]);
                    double y = s->u[d] + dt * s->v[d];
                    num += x * x;
                    den += y * y;
                    s->pu[d] = s->u[d];
                    s->pv[d] = s->v[d];
                }
        } else {
            for (int k = 0; k < s->r; ++k) {
                double x = (s->q[k] - s->pq[k]) + dt * (s->qd[k] - s->pqd[k]);
                double y = s->q[k] + dt * s->qd[k];
                num += x * x;
                den += y * y;
                s->pq[k] = s->q[k];
                s->pqd[k] = s->qd[k];
            }
        }
    }
    *cnum = num; *cden = den;
    *nonfinite = !(isfinite(num) && isfinite(den));
}

/* One controller step I_k (Algorithm 1): save, zero-order-hold initial boundary data, then
 * multiplicative (or additive) sweeps until the criterion holds at iteration n >= 2 or max_it is
 * reached. */
int orc_step(void* vp, int* iters, double* cnum_out, double* cden_out) {
    oprob* p = (oprob*)vp;
    if (!p->initialised) return ORC_EINVAL;
    save_state(p);
    /* zero-order hold of every source's state at t_{k-1} over all slots */
    for (int k = 0; k < p->ncpl; ++k) zoh(p, &p->cpl[k]);
    int n, status = ORC_MAXITER;
    double cnum = 0.0, cden = 0.0;
    for (n = 1; n <= p->max_it; ++n) {
        if (n > 1) restore_state(p);
        for (int i = 0; i < p->nsd; ++i) {
            advance(p, i);
            if (!p->additive) publish_from(p, i);
        }
        if (p->additive)
            for (int i = 0; i < p->nsd; ++i) publish_from(p, i);
        int nonfinite = 0;
        criterion(p, &cnum, &cden, &nonfinite);
        if (nonfinite) { status = ORC_ENONFINITE; break; }
        if (p->ncpl == 0) { status = ORC_OK; break; } /* a lone subdomain needs no Schwarz iteration */
        if (n >= 2 && (cnum < p->tol_abs * p->tol_abs || cnum < p->tol_rel * p->tol_rel * cden)) {
            status = ORC_OK;
            break;
        }
    }
    if (n > p->max_it) n = p->max_it;
    if (iters) *iters = n;
    if (cnum_out) *cnum_out = cnum;
    if (cden_out) *cden_out = cden;
    return status;
}

int orc_num_nodes(void* vp, int i) { return ((oprob*)vp)->sd[i].m.nn; }
int orc_num_free(void* vp, int i) { return ((oprob*)vp)->sd[i].nfree; }
int orc_num_schwarz(void* vp, int i) { return ((oprob*)vp)->sd[i].ns; }

/* FOM: copy (u, v, a); ROM: the reconstructed full fields (Phi q on free dofs, boundary data on
 * Schwarz dofs from the last slot, zero on clamped dofs).  Any output pointer may be NULL. */
int orc_get_state(void* vp, int i, double* u, double* v, double* a) {
    oprob* p = (oprob*)vp;
    osub* s = &p->sd[i];
    size_t n3 = 3 * (size_t)s->m.nn;
    if (s->kind == ORC_FOM) {
        if (u) memcpy(u, s->u, n3 * sizeof(double));
        if (v) memcpy(v, s->v, n3 * sizeof(double));
        if (a) memcpy(a, s->a, n3 * sizeof(double));
        return ORC_OK;
    }
    double* outs[3] = {u, v, a};
    const double* qs[3] = {s->q, s->qd, s->qdd};
    for (int f = 0; f < 3; ++f) {
        if (!outs[f]) continue;
        for (int n = 0; n < s->m.nn; ++n)
            for (int c = 0; c < 3; ++c) outs[f][3 * n + c] = rom_field(p, s, f, n, c, qs[f], s->nsub);
    }
    return ORC_OK;
}

int orc_get_rom(void* vp, int i, double* q, double* qd, double* qdd) {
    oprob* p = (oprob*)vp;
    osub* s = &p->sd[i];
    if (s->kind != ORC_ROM) return ORC_EINVAL;
    if (q) memcpy(q, s->q, sizeof(double) * s->r);
    if (qd) memcpy(qd, s->qd, sizeof(double) * s->r);
    if (qdd) memcpy(qdd, s->qdd, sizeof(double) * s->r);
    return ORC_OK;
}

/* Schwarz dof ids (3*node + c, increasing) and free dof ids of subdomain i */
int orc_schwarz_dofs(void* vp, int i, int* out) {
    osub* s = &((oprob*)vp)->sd[i];
    int t = 0;
    for (int r = 0; r < s->ns; ++r)
        for (int c = 0; c < 3; ++c) out[t++] = 3 * s->snode[r] + c;
    return t;
}

int orc_free_dofs(void* vp, int i, int* out) {
    osub* s = &((oprob*)vp)->sd[i];
    int t = 0;
    for (int n = 0; n < s->m.nn; ++n)
        for (int c = 0; c < 3; ++c)
            if (is_free(s, n, c)) out[t++] = 3 * n + c;
    return t;
}

/* ------------------------------------------------------------------------------------------ */
/* single-domain explicit rollout and its reverse-mode adjoint                                 */
/* ------------------------------------------------------------------------------------------ */
/* Forward: a0 = -M^-1 f(u0); per step u += dt v + dt^2/2 a; a' = -M^-1 f(u); v += dt/2 (a + a');
 * clamped components stay 0.  J = w . u_T.  Gradients of J w.r.t. u0, v0 and per-element
 * (lambda_e, mu_e) by the transposed recursion, storing every displacement (plain, no checkpointing). */
static void rollout(const omesh* m, int model, const double* lam_e, const double* mu_e, const double* mass,
                    const unsigned char* dmask, const double* u0, const double* v0, double dt, int nsteps,
                    double* ustore /* (nsteps+1)*3nn or NULL */, double* uT) {
    size_t n3 = 3 * (size_t)m->nn;
    double* u = dup_or_zero(u0, n3);
    double* v = dup_or_zero(v0, n3);
    double* a = dup_or_zero(NULL, n3);
    double* f = dup_or_zero(NULL, n3);
    for (size_t d = 0; d < n3; ++d)
        if (dmask[d / 3] & (1 << (d % 3))) { u[d] = 0.0; v[d] = 0.0; }
    internal_force(m, model, 0.0, 0.0, lam_e, mu_e, u, f);
    for (size_t d = 0; d < n3; ++d) a[d] = (dmask[d / 3] & (1 << (d % 3))) ? 0.0 : -f[d] / mass[d / 3];
    if (ustore) memcpy(ustore, u, n3 * sizeof(double));
    for (int t = 0; t < nsteps; ++t) {
        for (size_t d = 0; d < n3; ++d)
            if (!(dmask[d / 3] & (1 << (d % 3)))) u[d] += dt * v[d] + 0.5 * dt * dt * a[d];
        internal_force(m, model, 0.0, 0.0, lam_e, mu_e, u, f);
        for (size_t d = 0; d < n3; ++d) {
            if (dmask[d / 3] & (1 << (d % 3))) continue;
            double an = -f[d] / mass[d / 3];
            v[d] += 0.5 * dt * (a[d] + an);
            a[d] = an;
        }
        if (ustore) memcpy(ustore + (size_t)(t + 1) * n3, u, n3 * sizeof(double));
    }
    if (uT) memcpy(uT, u, n3 * sizeof(double));
    free(u); free(v); free(a); free(f);
}

int orc_rollout(int nx, int ny, int nz, double h, const double* org, int model, const double* lam_e,
                const double* mu_e, double rho, const unsigned char* dmask, const double* u0, const double* v0,
                double dt, int nsteps, double* uT) {
    omesh m;
    mesh_set(&m, nx, ny, nz, h, org);
    double* mass = dup_or_zero(NULL, (size_t)m.nn);
    lumped_mass(&m, rho, mass);
    rollout(&m, model, lam_e, mu_e, mass, dmask, u0, v0, dt, nsteps, NULL, uT);
    free(mass);
    return ORC_OK;
}

int orc_adjoint(int nx, int ny, int nz, double h, const double* org, int model, const double* lam_e,
                const double* mu_e, double rho, const unsigned char* dmask, const double* u0, const double* v0,
                double dt, int nsteps, const double* w, double* J, double* gu0, double* gv0, double* glam,
                double* gmu) {
    if (model == ORC_SVK) return ORC_EINVAL;
    omesh m;
    mesh_set(&m, nx, ny, nz, h, org);
    size_t n3 = 3 * (size_t)m.nn, ne = (size_t)m.ne;
    double* mass = dup_or_zero(NULL, (size_t)m.nn);
    lumped_mass(&m, rho, mass);
    double* us = (double*)malloc(sizeof(double) * n3 * (size_t)(nsteps + 1));
    if (!us) { free(mass); return ORC_ENOMEM; }
    rollout(&m, model, lam_e, mu_e, mass, dmask, u0, v0, dt, nsteps, us, NULL);
    double Jv = 0.0;
    for (size_t d = 0; d < n3; ++d) Jv += w[d] * us[(size_t)nsteps * n3 + d];
    *J = Jv;
    double* ub = dup_or_zero(w, n3);      /* adjoint of u_{n+1} (accumulating) */
    double* vb = dup_or_zero(NULL, n3);
    double* ab = dup_or_zero(NULL, n3);
    double* y = dup_or_zero(NULL, n3);
    double* tmp = dup_or_zero(NULL, n3);
    double* lb = dup_or_zero(NULL, ne);
    double* mb = dup_or_zero(NULL, ne);
    double* gl = dup_or_zero(NULL, ne);
    double* gm = dup_or_zero(NULL, ne);
    for (size_t d = 0; d < n3; ++d)
        if (dmask[d / 3] & (1 << (d % 3))) ub[d] = 0.0;
    for (int t = nsteps - 1; t >= 0; --t) {
        /* step t -> t+1.  v_{t+1} = v_t + dt/2 (a_t + a_{t+1}) */
        for (size_t d = 0; d < n3; ++d) ab[d] += 0.5 * dt * vb[d]; /* contribution to a_{t+1} */
        /* a_{t+1} = -M^-1 f(u_{t+1}) on free dofs */
        for (size_t d = 0; d < n3; ++d)
            y[d] = (dmask[d / 3] & (1 << (d % 3))) ? 0.0 : -ab[d] / mass[d / 3];
        force_vjp(&m, model, lam_e, mu_e, us + (size_t)(t + 1) * n3, y, tmp, lb, mb);
        for (size_t d = 0; d < n3; ++d)
            if (!(dmask[d / 3] & (1 << (d % 3)))) ub[d] += tmp[d];
        for (size_t e = 0; e < ne; ++e) { gl[e] += lb[e]; gm[e] += mb[e]; }
        /* now ub, vb hold the complete adjoints of u_{t+1}, v_{t+1}; a_{t+1}'s adjoint is consumed */
        double* ab_t = tmp;
        for (size_t d = 0; d < n3; ++d) {
            if (dmask[d / 3] & (1 << (d % 3))) { ab_t[d] = 0.0; continue; }
            /* v_{t+1} -> a_t, v_t ; u_{t+1} = u_t + dt v_t + dt^2/2 a_t */
            ab_t[d] = 0.5 * dt * vb[d] + 0.5 * dt * dt * ub[d];
            vb[d] = vb[d] + dt * ub[d];
            /* ub stays (du_{t+1}/du_t = I) */
        }
        memcpy(ab, ab_t, n3 * sizeof(double));
    }
    /* a_0 = -M^-1 f(u_0) */
    for (size_t d = 0; d < n3; ++d) y[d] = (dmask[d / 3] & (1 << (d % 3))) ? 0.0 : -ab[d] / mass[d / 3];
    force_vjp(&m, model, lam_e, mu_e, us, y, tmp, lb, mb);
    for (size_t d = 0; d < n3; ++d) {
        int clamped = dmask[d / 3] & (1 << (d % 3));
        gu0[d] = clamped ? 0.0 : ub[d] + tmp[d];
        gv0[d] = clamped ? 0.0 : vb[d];
    }
    for (size_t e = 0; e < ne; ++e) { glam[e] = gl[e] + lb[e]; gmu[e] = gm[e] + mb[e]; }
    free(us); free(mass); free(ub); free(vb); free(ab); free(y); free(tmp); free(lb); free(mb); free(gl); free(gm);
    return ORC_OK;
}
