// Internal declarations of libosam: device data of the subdomains and couplings, and the kernel
// launchers shared between translation units.  Not part of the public ABI (include/osam.h).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "osam.h"

namespace osam {

// element-to-node scatter of the internal force
enum Scatter { kAtomic = 1, kGather = 2 };

struct Grid {
    int nx = 0, ny = 0, nz = 0;
    double h = 0.0;
    double org[3] = {0, 0, 0};
    int nn() const { return (nx + 1) * (ny + 1) * (nz + 1); }
    int ne() const { return nx * ny * nz; }
};

// Arguments of the hex8 internal-force kernel.  Displacements are read at u[n*usn + c*usc];
// atomic mode adds into f[n*fsn + c*fsc]; gather mode writes the 24 element contributions to
// fe[(corner*3 + c)*ne + e], corner = ax + 2*ay + 4*az.
struct ElemArgs {
    int nx, ny, nz, ne;
    double invh, w8;          // 1/h and h^2/8 (Gauss weight x detJ / h for unit cubes)
    double lam, mu;
    const double* lam_e;
    const double* mu_e;
    const double* u;
    int usn;
    long long usc;
    void* f;
    int fsn;
    long long fsc;
    void* fe;
};

// Arguments of the node kernel that finishes substep j (corrector) and predicts substep j+1.
struct NodeArgs {
    int nx, ny, nz, nn, ne;
    double dt;
    const double* minv;       // 1 / lumped mass
    const uint8_t* clamp;     // per-node clamp bits
    const int* srow;          // per-node Schwarz row or -1
    int ns;                   // Schwarz rows
    const double* h1;         // history slot j+1: [3 fields][3 comps][ns]
    const double* h2;         // history slot j+2 (u field used) or null when j+1 is the last slot
    const double* ucur;       // u^{j+1}
    double* unext;            // out: u^{j+2} (unused when h2 == null and last)
    double* v;
    double* a;
    const void* force;        // f [3][nn] (atomic) or fe [24][ne] (gather)
    void* fclear;             // atomic mode: f array to reset to zero after reading
    int last;                 // 1 on the last substep of the interval (no predictor)
    int predict_only;         // 1: write unext = predictor of ucur with (v, a); no force used
};

struct FomDev {
    Grid g;
    int material = 0;
    double lam = 0, mu = 0, rho = 0;
    double* lam_e = nullptr;
    double* mu_e = nullptr;
    double* minv = nullptr;
    uint8_t* clamp = nullptr;
    int* srow = nullptr;
    int ns = 0;
    double* u[2] = {nullptr, nullptr};
    double* v = nullptr;
    double* a = nullptr;
    void* f = nullptr;        // atomic accumulation buffer [3][nn] (double or float)
    void* fe = nullptr;       // gather buffer [24][ne] (double or float)
    double* su = nullptr;
    double* sv = nullptr;
    double* sa = nullptr;
    double* pu = nullptr;
    double* pv = nullptr;
    double* hist = nullptr;   // input boundary history [(nsub+1)][3][3][ns]
    int norm_blocks = 0;
};

struct RomDev {
    Grid g;
    int r = 0, rs = 0, nfree = 0, nsdof = 0, d = 0, nq = 0;
    double* O = nullptr;       // packed operator [r][d] = [K | H | B | c]
    double* PhiSt = nullptr;   // Phi_S^T [rs][nsdof]
    double* Phi = nullptr;     // [nfree][r]
    int* free_dof = nullptr;   // [nfree] dof ids
    int* dof_free = nullptr;   // [3 nn] free row of each dof or -1
    uint8_t* clamp = nullptr;
    int* srow = nullptr;
    int ns = 0;
    short2* kron_ij = nullptr; // [nq] (i, j) of each compressed Kronecker entry
    double* q = nullptr;       // state [3][r] = q, qd, qdd
    double* sq = nullptr;      // saved [3][r]
    double* pq = nullptr;      // previous iterate [3][r]
    double* qrec = nullptr;    // recorded [(nsub+1)][3][r]
    double* ghat = nullptr;    // [(nsub+1)][rs]
    double* hist = nullptr;    // input boundary history [(nsub+1)][3][nsdof]
    double* partial = nullptr; // ROM step partial sums
    unsigned int* counter = nullptr;
    int step_gx = 0, step_gy = 0;
};

struct CplDev {
    int dst = 0, src = 0, nrow = 0;
    int nfield = 3;            // fields recorded / transferred (3, or 1 for a ROM destination's u... kept 3)
    int* row = nullptr;        // dst Schwarz row of each coupling row
    int* dnode = nullptr;      // [nrow][8] donor nodes in src
    double* dw = nullptr;      // [nrow][8] trilinear weights
    double* rec = nullptr;     // FOM source: recorded trace [(nsub+1)][3][3][nrow]
    double* Rt = nullptr;      // ROM source: (Pi Phi_rows)^T [r][3 nrow]
};

// ------------------------------------------------------------------------------------------------
// launchers (all asynchronous on `s`)
// ------------------------------------------------------------------------------------------------
cudaError_t launch_hex8_force(int material, bool fp32, int scatter, const ElemArgs& a, cudaStream_t s);
cudaError_t launch_node_update(bool fp32, int scatter, const NodeArgs& a, cudaStream_t s);
cudaError_t launch_lumped_minv(const Grid& g, double rho, double* minv, cudaStream_t s);
cudaError_t launch_trace(const CplDev& c, const double* u, const double* v, const double* a, int nn, int slot,
                         int nsub, cudaStream_t s);
cudaError_t launch_zoh_from_fom(const CplDev& c, const double* u, const double* v, const double* a, int nn,
                                bool dst_rom, double* dst_hist, int dst_ns_or_nsdof, int nsub, cudaStream_t s);
cudaError_t launch_publish_fom(const CplDev& c, bool dst_rom, double* dst_hist, int dst_ns_or_nsdof, int nsub,
                               cudaStream_t s);
cudaError_t launch_norms_fom(const FomDev& f, double dt, double* partial, cudaStream_t s);
cudaError_t launch_norms_final(const double* partial, int nparts, double* result, cudaStream_t s);
cudaError_t launch_donor(const Grid& src, const Grid& dst, const uint8_t* mask_dummy, const int* dst_nodes, int nrow,
                         int* dnode, double* dw, int* err, cudaStream_t s);
cudaError_t launch_gather_force(const Grid& g, const double* fe, double* f, cudaStream_t s);
cudaError_t launch_aos_to_soa(const double* aos, double* soa, int nn, cudaStream_t s);
cudaError_t launch_soa_to_aos(const double* soa, double* aos, int nn, cudaStream_t s);
cudaError_t launch_accel_from_force(const FomDev& f, const double* force_soa, cudaStream_t s);

// ROM
cudaError_t launch_rom_project(const RomDev& r, int slot0, int slot1, cudaStream_t s);
cudaError_t launch_rom_step(const RomDev& r, int slot, double dt, int rhs_only, cudaStream_t s);
cudaError_t launch_rom_reconstruct(const CplDev& c, const RomDev& src, bool zoh, bool dst_rom, double* dst_hist,
                                   int dst_ns_or_nsdof, int nsub, cudaStream_t s);
cudaError_t launch_rom_norms(const RomDev& r, double dt, double* partial, cudaStream_t s);
cudaError_t launch_rom_basis_project(const RomDev& r, const double* u_aos, const double* v_aos, cudaStream_t s);
cudaError_t launch_rom_full_field(const RomDev& r, const double* qv, int field, double* out_aos, int slot,
                                  cudaStream_t s);
cudaError_t launch_build_Rt_checked(const CplDev& c, const RomDev& src, int* err, cudaStream_t s);

// dense helpers (fit)
cudaError_t launch_gemm_tn(int m, int n, int k, const double* A, int lda, const double* B, int ldb, double* C,
                           int ldc, double alpha, double beta, cudaStream_t s);
cudaError_t launch_gemm_nn(int m, int n, int k, const double* A, int lda, const double* B, int ldb, double* C,
                           int ldc, double alpha, double beta, cudaStream_t s);
cudaError_t launch_gemm_nt(int m, int n, int k, const double* A, int lda, const double* B, int ldb, double* C,
                           int ldc, double alpha, double beta, cudaStream_t s);
cudaError_t launch_kron_features(const double* Ubar, int r, int nsnap, double* D, int ldd, int col0,
                                 cudaStream_t s);

// adjoint
cudaError_t launch_hex8_vjp(int material, const ElemArgs& a, const double* ybar, int ysn, long long ysc,
                            double* lam_bar, double* mu_bar, int accumulate, cudaStream_t s);
cudaError_t launch_adjoint_pre(int nn, double dt, const uint8_t* clamp, const double* minv, const double* vb, double* ab,
                               double* y, double* tmp, cudaStream_t s);
cudaError_t launch_adjoint_post(int nn, double dt, const uint8_t* clamp, const double* tmp, double* ub, double* vb,
                                double* ab, cudaStream_t s);
cudaError_t launch_zero_clamped(int nn, const uint8_t* clamp, double* u, double* v, cudaStream_t s);

int grid_for(long long n, int block);

// message returned by osam_last_error(NULL) on the calling thread
void set_thread_error(const std::string& msg);

}  // namespace osam
