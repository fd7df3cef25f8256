// opinf_fit: the offline OpInf stage of Sec. 3 and Sec. 4.2.1 (Eq. opinf_schwarz_inference).
//   POD by the method of snapshots: G = U U^T (n_snap x n_snap Gram, device GEMM over the long dof
//   dimension), G = V diag(sigma^2) V^T (Householder tridiagonalisation + implicit QL on the host),
//   Phi = U^T V_r Sigma_r^-1,
//   then one Cholesky re-orthonormalisation Phi <- Phi L^-T with L L^T = Phi^T Phi (same span).
//   Boundary basis Phi_S likewise from the Schwarz snapshots, r_s chosen by the energy criterion
//   (Eq. pod_energy: smallest r with E_r >= energy_s).
//   Regression: D = [Ubar^T, kron_c(Ubar)^T, Ghat^T, 1], Y = Abar^T, Tikhonov with one lambda,
//   dual form O = D^T (D D^T + lambda I)^-1 Y when D has more columns than rows, else the primal
//   normal equations (D^T D + lambda I) O = D^T Y; the small SPD systems are factored by Cholesky
//   on the host.
// opinf_select: Schwarz-aware regularisation selection (Sec. 4.2.4, Algorithm 3): the lambda-
//   independent part once, one Tikhonov solve per candidate, every candidate ROM rolled out on the
//   device under the frozen training boundary data (k_select_rollout, rom_kernels.cu), the minimiser
//   of Eq. schwarz_regularization_error returned with its operators.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "osam.h"
#include "osam_internal.h"

using namespace osam;

namespace {

thread_local std::string g_fit_error;

// Symmetric eigen-decomposition by Householder reduction to tridiagonal form followed by the
// implicit QL iteration with Wilkinson-type shifts (Householder 1958; Bowdler, Martin, Reinsch and
// Wilkinson 1968).  A is n x n, row-major, symmetric; on return A's diagonal holds the eigenvalues
// and V (row-major) the eigenvectors as columns.  About 9 n^3 flops with contiguous row access.
void sym_eig(std::vector<double>& A, int n, std::vector<double>& V) {
    std::vector<double> d(n), e(n, 0.0), tau(n, 0.0), p(n), w(n);
    // (1) A <- H_k A H_k, H_k = I - tau_k v_k v_k^T acting on rows / columns k+1..n-1; v_k is kept in
    //     row k to the right of the diagonal (the part of A that the reduction no longer needs)
    for (int k = 0; k + 2 < n; ++k) {
        double* ak = &A[(size_t)k * n];
        const int m0 = k + 1;
        double scale = 0.0;
        for (int i = m0; i < n; ++i) scale = std::max(scale, std::fabs(ak[i]));
        if (scale == 0.0) { e[k] = 0.0; tau[k] = 0.0; continue; }
        double ss = 0.0;
        for (int i = m0; i < n; ++i) { ak[i] /= scale; ss += ak[i] * ak[i]; }
        const double nrm = std::sqrt(ss);
        const double alpha = ak[m0] > 0.0 ? -nrm : nrm;      // reflect x onto alpha e_1
        e[k] = alpha * scale;
        ak[m0] -= alpha;                                     // v = x - alpha e_1
        const double vv = ss - 2.0 * alpha * (ak[m0] + alpha) + alpha * alpha;  // |v|^2
        const double t = vv > 0.0 ? 2.0 / vv : 0.0;
        tau[k] = t;
        // p = t B v with B = A[m0.., m0..] (symmetric: use rows), then w = p - (t/2)(p.v) v
        for (int i = m0; i < n; ++i) {
            const double* ai = &A[(size_t)i * n];
            double s = 0.0;
            for (int j = m0; j < n; ++j) s += ai[j] * ak[j];
            p[i] = t * s;
        }
        double pv = 0.0;
        for (int i = m0; i < n; ++i) pv += p[i] * ak[i];
        const double kk = 0.5 * t * pv;
        for (int i = m0; i < n; ++i) w[i] = p[i] - kk * ak[i];
        // B <- B - v w^T - w v^T
        for (int i = m0; i < n; ++i) {
            double* ai = &A[(size_t)i * n];
            const double vi = ak[i], wi = w[i];
            for (int j = m0; j < n; ++j) ai[j] -= vi * w[j] + wi * ak[j];
        }
    }
    for (int k = 0; k < n; ++k) d[k] = A[(size_t)k * n + k];
    if (n >= 2) e[n - 2] = A[(size_t)(n - 2) * n + (n - 1)];
    // (2) Q = H_0 H_1 ... H_{n-3}, accumulated from the last reflector; Z = Q^T (rows = vectors)
    std::vector<double> Q((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
    for (int k = n - 3; k >= 0; --k) {
        const double t = tau[k];
        if (t == 0.0) continue;
        const double* v = &A[(size_t)k * n];
        const int m0 = k + 1;
        // Q[m0.., m0..] <- (I - t v v^T) Q[m0.., m0..]: s_j = t sum_i v_i Q_ij, Q_ij -= v_i s_j
        std::fill(p.begin(), p.end(), 0.0);
        for (int i = m0; i < n; ++i) {
            const double vi = v[i];
            const double* qi = &Q[(size_t)i * n];
            for (int j = m0; j < n; ++j) p[j] += vi * qi[j];
        }
        for (int i = m0; i < n; ++i) {
            const double vi = t * v[i];
            double* qi = &Q[(size_t)i * n];
            for (int j = m0; j < n; ++j) qi[j] -= vi * p[j];
        }
    }
    std::vector<double> Z((size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Z[(size_t)j * n + i] = Q[(size_t)i * n + j];
    // (3) implicit QL on (d, e), e[i] coupling d[i] and d[i+1]; each plane rotation of rows i, i+1 of
    //     the tridiagonal matrix is applied to rows i, i+1 of Z
    for (int l = 0; l < n; ++l) {
        for (int iter = 0; iter < 60; ++iter) {
            int m = l;
            for (; m + 1 < n; ++m) {
                const double dd = std::fabs(d[m]) + std::fabs(d[m + 1]);
                if (std::fabs(e[m]) <= 1e-16 * dd) break;
            }
            if (m == l) break;
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double r = std::hypot(g, 1.0);
            g = d[m] - d[l] + e[l] / (g + (g >= 0.0 ? r : -r));   // shifted so that the shift is the
            double s = 1.0, c = 1.0, pp = 0.0;                     // eigenvalue of the leading 2x2 closer to d[l]
            int i = m - 1;
            bool deflated = false;
            for (; i >= l; --i) {
                const double f = s * e[i], b = c * e[i];
                r = std::hypot(f, g);
                e[i + 1] = r;
                if (r == 0.0) { d[i + 1] -= pp; e[m] = 0.0; deflated = true; break; }
                s = f / r;
                c = g / r;
                g = d[i + 1] - pp;
                r = (d[i] - g) * s + 2.0 * c * b;
                pp = s * r;
                d[i + 1] = g + pp;
                g = c * r - b;
                double* zi = &Z[(size_t)i * n];
                double* zj = &Z[(size_t)(i + 1) * n];
                for (int k = 0; k < n; ++k) {
                    const double a0 = zi[k], a1 = zj[k];
                    zj[k] = s * a0 + c * a1;
                    zi[k] = c * a0 - s * a1;
                }
            }
            if (deflated) continue;
            d[l] -= pp;
            e[l] = g;
            e[m] = 0.0;
        }
    }
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) V[(size_t)k * n + i] = Z[(size_t)i * n + k];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) A[(size_t)i * n + j] = i == j ? d[i] : 0.0;
}

// Cholesky L L^T = A (row-major, lower triangle written into A); false if not positive definite
bool cholesky(std::vector<double>& A, int n) {
    for (int j = 0; j < n; ++j) {
        double s = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) s -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
        if (!(s > 0.0)) return false;
        const double d = std::sqrt(s);
        A[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double t = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) t -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
            A[(size_t)i * n + j] = t / d;
        }
    }
    return true;
}

// solve L L^T X = B in place (B row-major n x m)
void chol_solve(const std::vector<double>& L, int n, std::vector<double>& B, int m) {
    for (int c = 0; c < m; ++c) {
        for (int i = 0; i < n; ++i) {
            double t = B[(size_t)i * m + c];
            for (int k = 0; k < i; ++k) t -= L[(size_t)i * n + k] * B[(size_t)k * m + c];
            B[(size_t)i * m + c] = t / L[(size_t)i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {
            double t = B[(size_t)i * m + c];
            for (int k = i + 1; k < n; ++k) t -= L[(size_t)k * n + i] * B[(size_t)k * m + c];
            B[(size_t)i * m + c] = t / L[(size_t)i * n + i];
        }
    }
}

struct Dev {
    std::vector<void*> ptrs;
    ~Dev() { for (void* p : ptrs) cudaFree(p); }
    double* alloc(size_t n) {
        void* p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(double)) != cudaSuccess) return nullptr;
        ptrs.push_back(p);
        return static_cast<double*>(p);
    }
};

#define FK(call)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            g_fit_error = std::string(#call) + ": " + cudaGetErrorString(e_);      \
            return OSAM_ECUDA;                                                     \
        }                                                                          \
    } while (0)
#define FA(p)                                                       \
    do {                                                            \
        if (!(p)) { g_fit_error = "device allocation failed"; return OSAM_ENOMEM; } \
    } while (0)

// POD of snapshots X [n_snap][n] on the device: returns Phi [n][r] (device), sigma (host, all).
// r > 0 fixes the rank; r <= 0 selects the smallest rank whose energy E_r reaches `energy`, capped
// at r_max; the rank used is returned in *r_used.
int pod(cudaStream_t s, Dev& dev, const double* X, int nsnap, int n, int r, double energy, int r_max,
        int* r_used, double** Phi_out, std::vector<double>& sigma) {
    double* G = dev.alloc((size_t)nsnap * nsnap);
    FA(G);
    FK(launch_gemm_nt(nsnap, nsnap, n, X, n, X, n, G, nsnap, 1.0, 0.0, s));
    std::vector<double> Gh((size_t)nsnap * nsnap), V;
    FK(cudaMemcpyAsync(Gh.data(), G, sizeof(double) * Gh.size(), cudaMemcpyDeviceToHost, s));
    FK(cudaStreamSynchronize(s));
    for (int i = 0; i < nsnap; ++i)  // exact symmetry
        for (int j = i + 1; j < nsnap; ++j) Gh[(size_t)j * nsnap + i] = Gh[(size_t)i * nsnap + j];
    sym_eig(Gh, nsnap, V);
    std::vector<int> order(nsnap);
    for (int i = 0; i < nsnap; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return Gh[(size_t)a * nsnap + a] > Gh[(size_t)b * nsnap + b]; });
    sigma.resize(nsnap);
    for (int i = 0; i < nsnap; ++i) sigma[i] = std::sqrt(std::max(0.0, Gh[(size_t)order[i] * nsnap + order[i]]));
    if (r <= 0) {
        double tot = 0.0, acc = 0.0;
        for (double x : sigma) tot += x * x;
        r = nsnap;
        for (int k = 0; k < nsnap; ++k) {
            acc += sigma[k] * sigma[k];
            if (acc >= energy * tot) { r = k + 1; break; }
        }
        if (r_max > 0) r = std::min(r, r_max);
        while (r > 1 && !(sigma[r - 1] > 0.0)) --r;
    }
    *r_used = r;
    if (r > nsnap) { g_fit_error = "POD rank exceeds the snapshot count"; return OSAM_EINVAL; }
    if (r > 0 && !(sigma[r - 1] > 0.0)) { g_fit_error = "snapshot matrix rank is below the requested POD rank"; return OSAM_EINVAL; }
    // W = V_r Sigma_r^-1 [nsnap][r]
    std::vector<double> W((size_t)nsnap * r);
    for (int i = 0; i < nsnap; ++i)
        for (int k = 0; k < r; ++k) W[(size_t)i * r + k] = V[(size_t)i * nsnap + order[k]] / sigma[k];
    double* Wd = dev.alloc(W.size());
    double* Phi = dev.alloc((size_t)n * r);
    FA(Wd); FA(Phi);
    FK(cudaMemcpyAsync(Wd, W.data(), sizeof(double) * W.size(), cudaMemcpyHostToDevice, s));
    FK(launch_gemm_tn(n, r, nsnap, X, n, Wd, r, Phi, r, 1.0, 0.0, s));
    // re-orthonormalise: M = Phi^T Phi = L L^T, Phi <- Phi L^-T
    double* M = dev.alloc((size_t)r * r);
    FA(M);
    FK(launch_gemm_tn(r, r, n, Phi, r, Phi, r, M, r, 1.0, 0.0, s));
    std::vector<double> Mh((size_t)r * r);
    FK(cudaMemcpyAsync(Mh.data(), M, sizeof(double) * Mh.size(), cudaMemcpyDeviceToHost, s));
    FK(cudaStreamSynchronize(s));
    if (!cholesky(Mh, r)) { g_fit_error = "POD basis re-orthonormalisation failed"; return OSAM_EINVAL; }
    // Linv^T (upper) as a dense r x r matrix: Phi_new = Phi * Linv^T
    std::vector<double> Li((size_t)r * r, 0.0);
    for (int c = 0; c < r; ++c) {  // solve L x = e_c
        for (int i = 0; i < r; ++i) {
            double t = (i == c) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) t -= Mh[(size_t)i * r + k] * Li[(size_t)k * r + c];
            Li[(size_t)i * r + c] = t / Mh[(size_t)i * r + i];
        }
    }
    std::vector<double> LiT((size_t)r * r);
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < r; ++j) LiT[(size_t)i * r + j] = Li[(size_t)j * r + i];
    double* T = dev.alloc((size_t)r * r);
    double* Phi2 = dev.alloc((size_t)n * r);
    FA(T); FA(Phi2);
    FK(cudaMemcpyAsync(T, LiT.data(), sizeof(double) * LiT.size(), cudaMemcpyHostToDevice, s));
    FK(launch_gemm_nn(n, r, r, Phi, r, T, r, Phi2, r, 1.0, 0.0, s));
    *Phi_out = Phi2;
    return OSAM_OK;
}

// The lambda-independent part of the fit: bases, projections, the data matrix and the Gram matrix of
// the regression (dual D D^T or primal D^T D, without lambda).
struct FitData {
    int ns = 0, n = 0, nsd = 0, r = 0, rs = 0, nq = 0, nc = 0, d = 0;
    bool dual = false;
    double* Phi = nullptr;    // device [n][r]
    double* PhiS = nullptr;   // device [nsd][rs]
    double* D = nullptr;      // device [ns][d] = [Ubar^T | kron_c(Ubar)^T | kron3_c(Ubar)^T | Ghat^T | 1]
    double* Y = nullptr;      // device [ns][r] = Abar^T
    std::vector<double> Yh;   // host Abar^T
    std::vector<double> M0;   // host Gram without lambda: [ns][ns] (dual) or [d][d] (primal)
    std::vector<double> R0;   // host D^T Y [d][r] (primal)
    std::vector<double> sigma, sigma_s;
};

// A snapshot matrix already in this device's memory is read in place (the fit never writes its
// inputs); host memory, or another device's, is copied into a buffer of the fit.
int snapshot_operand(const double* src, size_t count, int device, cudaStream_t s, Dev& dev, const double** out) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, src) == cudaSuccess && at.device == device &&
        (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)) {
        *out = src;
        return OSAM_OK;
    }
    cudaGetLastError();   // an unregistered host pointer may leave an error behind on older runtimes
    double* d = dev.alloc(count);
    FA(d);
    FK(cudaMemcpyAsync(d, src, sizeof(double) * count, cudaMemcpyDefault, s));
    *out = d;
    return OSAM_OK;
}

int fit_prepare(const osam_fit_input* in, cudaStream_t s, Dev& dev, FitData& F) {
    const int ns = in->n_snap, n = in->n_dof, nsd = in->n_sdof, r = in->r;
    F.ns = ns; F.n = n; F.nsd = nsd; F.r = r;
    const double* U = nullptr;
    const double* A = nullptr;
    if (int rc = snapshot_operand(in->U, (size_t)ns * n, in->device, s, dev, &U)) return rc;
    if (int rc = snapshot_operand(in->A, (size_t)ns * n, in->device, s, dev, &A)) return rc;
    int r_used = 0;
    if (int rc = pod(s, dev, U, ns, n, r, 0.0, 0, &r_used, &F.Phi, F.sigma)) return rc;
    // boundary basis
    const double* S = nullptr;
    if (nsd > 0) {
        if (int rc = snapshot_operand(in->S, (size_t)ns * nsd, in->device, s, dev, &S)) return rc;
        const int rs_cap = std::min(in->r_s_max > 0 ? in->r_s_max : ns, ns);
        if (int rc = pod(s, dev, S, ns, nsd, in->r_s > 0 ? std::min(in->r_s, ns) : 0, in->energy_s, rs_cap, &F.rs,
                         &F.PhiS, F.sigma_s))
            return rc;
    }
    const int rs = F.rs;
    const int nq = (in->quadratic || in->cubic) ? r * (r + 1) / 2 : 0;
    const int nc = in->cubic ? r * (r + 1) * (r + 2) / 6 : 0;
    const int d = r + nq + nc + rs + 1;
    F.nq = nq; F.nc = nc; F.d = d;
    // D [ns][d]
    double* D = dev.alloc((size_t)ns * d);
    double* Ubt = dev.alloc((size_t)ns * r);   // Ubar^T [ns][r]
    double* Ub = dev.alloc((size_t)r * ns);    // Ubar [r][ns]
    double* Y = dev.alloc((size_t)ns * r);     // Abar^T
    FA(D); FA(Ubt); FA(Ub); FA(Y);
    FK(launch_gemm_nn(ns, r, n, U, n, F.Phi, r, Ubt, r, 1.0, 0.0, s));
    FK(launch_gemm_nn(ns, r, n, A, n, F.Phi, r, Y, r, 1.0, 0.0, s));
    std::vector<double> Ubt_h((size_t)ns * r), Ub_h((size_t)r * ns);
    FK(cudaMemcpyAsync(Ubt_h.data(), Ubt, sizeof(double) * Ubt_h.size(), cudaMemcpyDeviceToHost, s));
    FK(cudaStreamSynchronize(s));
    for (int i = 0; i < ns; ++i)
        for (int k = 0; k < r; ++k) Ub_h[(size_t)k * ns + i] = Ubt_h[(size_t)i * r + k];
    FK(cudaMemcpyAsync(Ub, Ub_h.data(), sizeof(double) * Ub_h.size(), cudaMemcpyHostToDevice, s));
    std::vector<double> Dh((size_t)ns * d, 0.0);
    // linear block and constant on the host (small); Kronecker block and boundary block on the device
    FK(cudaMemsetAsync(D, 0, sizeof(double) * ns * d, s));
    if (nq) FK(launch_kron_features(Ub, r, ns, D, d, r, s));
    if (nc) FK(launch_kron3_features(Ub, r, ns, D, d, r + nq, s));
    if (rs) FK(launch_gemm_nn(ns, rs, nsd, S, nsd, F.PhiS, rs, D + r + nq + nc, d, 1.0, 0.0, s));
    FK(cudaMemcpyAsync(Dh.data(), D, sizeof(double) * Dh.size(), cudaMemcpyDeviceToHost, s));
    FK(cudaStreamSynchronize(s));
    for (int i = 0; i < ns; ++i) {
        for (int k = 0; k < r; ++k) Dh[(size_t)i * d + k] = Ubt_h[(size_t)i * r + k];
        Dh[(size_t)i * d + d - 1] = 1.0;
    }
    FK(cudaMemcpyAsync(D, Dh.data(), sizeof(double) * Dh.size(), cudaMemcpyHostToDevice, s));
    F.Yh.resize((size_t)ns * r);
    FK(cudaMemcpyAsync(F.Yh.data(), Y, sizeof(double) * F.Yh.size(), cudaMemcpyDeviceToHost, s));
    FK(cudaStreamSynchronize(s));
    F.D = D;
    F.Y = Y;
    F.dual = d > ns;
    if (F.dual) {
        double* M = dev.alloc((size_t)ns * ns);
        FA(M);
        FK(launch_gemm_nt(ns, ns, d, D, d, D, d, M, ns, 1.0, 0.0, s));
        F.M0.resize((size_t)ns * ns);
        FK(cudaMemcpyAsync(F.M0.data(), M, sizeof(double) * F.M0.size(), cudaMemcpyDeviceToHost, s));
        FK(cudaStreamSynchronize(s));
        for (int i = 0; i < ns; ++i)
            for (int j = i + 1; j < ns; ++j) F.M0[(size_t)j * ns + i] = F.M0[(size_t)i * ns + j];
    } else {
        double* M = dev.alloc((size_t)d * d);
        double* R = dev.alloc((size_t)d * r);
        FA(M); FA(R);
        FK(launch_gemm_tn(d, d, ns, D, d, D, d, M, d, 1.0, 0.0, s));
        FK(launch_gemm_tn(d, r, ns, D, d, Y, r, R, r, 1.0, 0.0, s));
        F.M0.resize((size_t)d * d);
        F.R0.resize((size_t)d * r);
        FK(cudaMemcpyAsync(F.M0.data(), M, sizeof(double) * F.M0.size(), cudaMemcpyDeviceToHost, s));
        FK(cudaMemcpyAsync(F.R0.data(), R, sizeof(double) * F.R0.size(), cudaMemcpyDeviceToHost, s));
        FK(cudaStreamSynchronize(s));
        for (int i = 0; i < d; ++i)
            for (int j = i + 1; j < d; ++j) F.M0[(size_t)j * d + i] = F.M0[(size_t)i * d + j];
    }
    return OSAM_OK;
}

// Tikhonov solution for one lambda: O [d][r] (host)
int fit_solve(const FitData& F, double lambda, cudaStream_t s, Dev& dev, std::vector<double>& Oh) {
    const int ns = F.ns, d = F.d, r = F.r;
    Oh.assign((size_t)d * r, 0.0);
    if (F.dual) {
        // (D D^T + lambda I) Z = Y, O = D^T Z
        std::vector<double> Mh = F.M0, Zh = F.Yh;
        for (int i = 0; i < ns; ++i) Mh[(size_t)i * ns + i] += lambda;
        if (!cholesky(Mh, ns)) { g_fit_error = "regularised dual system is not positive definite"; return OSAM_EINVAL; }
        chol_solve(Mh, ns, Zh, r);
        double* Z = dev.alloc((size_t)ns * r);
        double* Od = dev.alloc((size_t)d * r);
        FA(Z); FA(Od);
        FK(cudaMemcpyAsync(Z, Zh.data(), sizeof(double) * Zh.size(), cudaMemcpyHostToDevice, s));
        FK(launch_gemm_tn(d, r, ns, F.D, d, Z, r, Od, r, 1.0, 0.0, s));
        FK(cudaMemcpyAsync(Oh.data(), Od, sizeof(double) * Oh.size(), cudaMemcpyDeviceToHost, s));
        FK(cudaStreamSynchronize(s));
    } else {
        std::vector<double> Mh = F.M0;
        Oh = F.R0;
        for (int i = 0; i < d; ++i) Mh[(size_t)i * d + i] += lambda;
        if (!cholesky(Mh, d)) { g_fit_error = "regularised normal equations are not positive definite"; return OSAM_EINVAL; }
        chol_solve(Mh, d, Oh, r);
    }
    return OSAM_OK;
}

// write the operators of O [d][r] and the bases to the caller's output
int fit_output(const osam_fit_input* in, const FitData& F, const std::vector<double>& Oh, cudaStream_t s,
               osam_fit_output* out) {
    const int r = F.r, nq = F.nq, nc = F.nc, rs = F.rs, d = F.d, nsd = F.nsd, ns = F.ns;
    const int nq_full = r * (r + 1) / 2;
    const int rs_cols = std::max(in->r_s_max, rs);
    std::vector<double> K((size_t)r * r), H((size_t)r * nq_full, 0.0), B((size_t)r * std::max(1, rs_cols), 0.0), c(r);
    std::vector<double> Cc((size_t)r * nc);
    for (int i = 0; i < r; ++i) {
        for (int k = 0; k < r; ++k) K[(size_t)i * r + k] = Oh[(size_t)k * r + i];
        for (int k = 0; k < nq; ++k) H[(size_t)i * nq_full + k] = Oh[(size_t)(r + k) * r + i];
        for (int k = 0; k < nc; ++k) Cc[(size_t)i * nc + k] = Oh[(size_t)(r + nq + k) * r + i];
        for (int k = 0; k < rs; ++k) B[(size_t)i * rs_cols + k] = Oh[(size_t)(r + nq + nc + k) * r + i];
        c[i] = Oh[(size_t)(d - 1) * r + i];
    }
    if (out->C && nc) FK(cudaMemcpyAsync(out->C, Cc.data(), sizeof(double) * Cc.size(), cudaMemcpyDefault, s));
    if (out->K) FK(cudaMemcpyAsync(out->K, K.data(), sizeof(double) * K.size(), cudaMemcpyDefault, s));
    if (out->H) FK(cudaMemcpyAsync(out->H, H.data(), sizeof(double) * H.size(), cudaMemcpyDefault, s));
    if (out->B && rs_cols > 0) FK(cudaMemcpyAsync(out->B, B.data(), sizeof(double) * (size_t)r * rs_cols, cudaMemcpyDefault, s));
    if (out->c) FK(cudaMemcpyAsync(out->c, c.data(), sizeof(double) * r, cudaMemcpyDefault, s));
    if (out->Phi) FK(cudaMemcpyAsync(out->Phi, F.Phi, sizeof(double) * (size_t)F.n * r, cudaMemcpyDefault, s));
    if (out->Phi_S && rs > 0) {
        // [nsd][rs] -> [nsd][rs_cols]
        std::vector<double> P((size_t)nsd * rs), Pw((size_t)nsd * rs_cols, 0.0);
        FK(cudaMemcpyAsync(P.data(), F.PhiS, sizeof(double) * P.size(), cudaMemcpyDeviceToHost, s));
        FK(cudaStreamSynchronize(s));
        for (int m = 0; m < nsd; ++m)
            for (int k = 0; k < rs; ++k) Pw[(size_t)m * rs_cols + k] = P[(size_t)m * rs + k];
        FK(cudaMemcpyAsync(out->Phi_S, Pw.data(), sizeof(double) * Pw.size(), cudaMemcpyDefault, s));
    }
    if (out->sigma) FK(cudaMemcpyAsync(out->sigma, F.sigma.data(), sizeof(double) * ns, cudaMemcpyDefault, s));
    if (out->sigma_s && !F.sigma_s.empty())
        FK(cudaMemcpyAsync(out->sigma_s, F.sigma_s.data(), sizeof(double) * ns, cudaMemcpyDefault, s));
    FK(cudaStreamSynchronize(s));
    out->r_s = rs;
    return OSAM_OK;
}

// The kernels of the fit index rows, snapshot columns and feature columns with 32-bit integers.
constexpr long long kFitMaxRows = 0x7fffffffLL - 64;

int fit_check(const osam_fit_input* in) {
    if (!in || !in->U || !in->A || in->n_dof < 1 || in->n_snap < 1 || in->r < 1 || in->r > 256 ||
        (in->n_sdof > 0 && !in->S) || (in->cubic && in->r > 128))
        return OSAM_EINVAL;
    if (in->n_dof > kFitMaxRows || in->n_sdof > kFitMaxRows || in->n_snap > kFitMaxRows) {
        g_fit_error = "n_dof, n_sdof and n_snap must be below 2^31 - 64";
        return OSAM_EINVAL;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) { g_fit_error = "no CUDA device"; return OSAM_ECUDA; }
    FK(cudaSetDevice(in->device));
    return OSAM_OK;
}

}  // namespace

extern "C" OSAM_API int opinf_fit(const osam_fit_input* in, osam_fit_output* out) {
    g_fit_error.clear();
    if (!out || !in || in->lambda < 0.0) return OSAM_EINVAL;
    if (int rc = fit_check(in)) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(in->stream);
    Dev dev;
    FitData F;
    if (int rc = fit_prepare(in, s, dev, F)) return rc;
    std::vector<double> Oh;
    if (int rc = fit_solve(F, in->lambda, s, dev, Oh)) return rc;
    return fit_output(in, F, Oh, s, out);
}

extern "C" OSAM_API int opinf_select(const osam_fit_input* in, const osam_select_input* sel, double* errors,
                                     int* best, osam_fit_output* out) {
    g_fit_error.clear();
    if (!out || !in || !sel || !sel->lambdas || sel->n_lambda < 1 || sel->n_lambda > 64 || !(sel->dt > 0.0) ||
        sel->substeps < 1 || !errors || !best)
        return OSAM_EINVAL;
    for (int l = 0; l < sel->n_lambda; ++l)
        if (!(sel->lambdas[l] >= 0.0)) return OSAM_EINVAL;
    if (in->r > 128) { g_fit_error = "regularisation selection supports r <= 128"; return OSAM_EINVAL; }
    if (int rc = fit_check(in)) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(in->stream);
    Dev dev;
    FitData F;
    if (int rc = fit_prepare(in, s, dev, F)) return rc;
    const int nl = sel->n_lambda, r = F.r, d = F.d;
    // packed operator rows [nl][r][d] (K | H | C | B | c), one fit per candidate
    std::vector<double> Op((size_t)nl * r * d);
    std::vector<std::vector<double>> Os(nl);
    for (int l = 0; l < nl; ++l) {
        if (int rc = fit_solve(F, sel->lambdas[l], s, dev, Os[l])) return rc;
        for (int i = 0; i < r; ++i)
            for (int k = 0; k < d; ++k) Op[((size_t)l * r + i) * d + k] = Os[l][(size_t)k * r + i];
    }
    std::vector<short2> kij;
    for (int i = 0; i < r; ++i)
        for (int j = i; j < r; ++j) kij.push_back(make_short2((short)i, (short)j));
    std::vector<short4> kijk;
    if (F.nc)
        for (int i = 0; i < r; ++i)
            for (int j = i; j < r; ++j)
                for (int k = j; k < r; ++k) kijk.push_back(make_short4((short)i, (short)j, (short)k, 0));
    double* Od = dev.alloc(Op.size());
    double* qd0 = dev.alloc(r);
    double* v0 = dev.alloc(F.n);
    double* phi = dev.alloc((size_t)nl * d);
    double* num = dev.alloc(nl);
    double* den = dev.alloc(nl);
    FA(Od); FA(qd0); FA(v0); FA(phi); FA(num); FA(den);
    short2* kd = nullptr;
    if (!kij.empty()) {
        if (cudaMalloc(&kd, sizeof(short2) * kij.size()) != cudaSuccess) { g_fit_error = "device allocation failed"; return OSAM_ENOMEM; }
        dev.ptrs.push_back(kd);
        FK(cudaMemcpyAsync(kd, kij.data(), sizeof(short2) * kij.size(), cudaMemcpyHostToDevice, s));
    }
    short4* kkd = nullptr;
    if (!kijk.empty()) {
        if (cudaMalloc(&kkd, sizeof(short4) * kijk.size()) != cudaSuccess) { g_fit_error = "device allocation failed"; return OSAM_ENOMEM; }
        dev.ptrs.push_back(kkd);
        FK(cudaMemcpyAsync(kkd, kijk.data(), sizeof(short4) * kijk.size(), cudaMemcpyHostToDevice, s));
    }
    FK(cudaMemcpyAsync(Od, Op.data(), sizeof(double) * Op.size(), cudaMemcpyHostToDevice, s));
    // qd0 = Phi^T v0
    if (sel->v0) {
        FK(cudaMemcpyAsync(v0, sel->v0, sizeof(double) * F.n, cudaMemcpyDefault, s));
        FK(launch_gemm_tn(r, 1, F.n, F.Phi, r, v0, 1, qd0, 1, 1.0, 0.0, s));
    } else {
        FK(cudaMemsetAsync(qd0, 0, sizeof(double) * r, s));
    }
    FK(launch_select_rollout(nl, r, d, F.nq, F.nc, F.rs, Od, kd, kkd, F.D, F.Y, qd0, F.ns, sel->substeps, sel->dt, phi, num,
                             den, s));
    std::vector<double> nh(nl), dh(nl);
    FK(cudaMemcpyAsync(nh.data(), num, sizeof(double) * nl, cudaMemcpyDeviceToHost, s));
    FK(cudaMemcpyAsync(dh.data(), den, sizeof(double) * nl, cudaMemcpyDeviceToHost, s));
    FK(cudaStreamSynchronize(s));
    int b = -1;
    for (int l = 0; l < nl; ++l) {
        const double e = std::sqrt(nh[l] / dh[l]);
        errors[l] = std::isfinite(e) ? e : HUGE_VAL;
        if (std::isfinite(e) && (b < 0 || e < errors[b])) b = l;
    }
    if (b < 0) { g_fit_error = "every candidate rollout is non-finite"; return OSAM_ENONFINITE; }
    *best = b;
    return fit_output(in, F, Os[b], s, out);
}

extern "C" OSAM_API const char* osam_fit_last_error(void) { return g_fit_error.c_str(); }

extern "C" OSAM_API int osam_fit_profile(int enable, double* gemm_ms, double* gemm_flops, long long* gemm_launches) {
    return osam::gemm_profile(enable, gemm_ms, gemm_flops, gemm_launches);
}
