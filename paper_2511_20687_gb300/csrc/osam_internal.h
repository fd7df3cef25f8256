// Internal declarations of libosam: device-side views of the batched subdomain groups and
// couplings, and the kernel launchers shared between translation units.  Not part of the public ABI
// (include/osam.h).
//
// A context holds n_inst instances of one coupled problem (same subdomain kinds, same coupling
// topology, same time step and substep count; meshes, materials and ROM operators may differ).
// Subdomain slot s of every instance forms one group whose arrays are concatenated across instances;
// per-instance tables give each instance's sizes and offsets, and block tables map every CUDA block
// of a per-step kernel to one instance, so a single launch advances every instance.  A single
// problem is a batch of one.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "osam.h"

namespace osam {

// element-to-node scatter of the internal force
enum Scatter { kAtomic = 1, kGather = 2 };

constexpr int kMaxSlots = 8;    // subdomains per instance
constexpr int kLinPerGp = 22;   // doubles per Gauss point of the stored Neo-Hookean Newton linearisation
constexpr int kNodeBlock = 128; // nodes per block of the node kernels

struct Grid {
    int nx = 0, ny = 0, nz = 0;
    double h = 0.0;
    double org[3] = {0, 0, 0};
    int nn() const { return (nx + 1) * (ny + 1) * (nz + 1); }
    int ne() const { return nx * ny * nz; }
};

// Arguments of the element-level hex8 kernel (one mesh).  Displacements are read at
// u[n*usn + c*usc]; atomic mode adds into f[n*fsn + c*fsc]; gather mode writes the 24 element
// contributions to fe[(corner*3 + c)*ne + e], corner = ax + 2*ay + 4*az.
struct ElemArgs {
    int nx, ny, nz, ne;
    double invh, w8;          // 1/h and h^2/8 (Gauss weight x detJ / h for unit cubes)
    double wq, wq3;           // h^2/32 and h^2/96 (the element force's material-factor weights)
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

// one instance of a FOM slot
struct InstFom {
    int nx, ny, nz, nn, ne, ns;
    double invh, w8, lam, mu;
    double wq, wq3;           // h^2/32 and h^2/96: weights of the force kernels' material factors
    double m1, m2, m3;        // material factors of the uniform material (hex8::material_factors)
    const double* lam_e;      // absolute device pointers or null (uniform lam / mu)
    const double* mu_e;
    long long node_off, elem_off, hist_off;
};

// kernel view of a FOM slot across instances; nodal arrays are SoA over the concatenated nodes:
// component c of global node g is at [c * NN + g]; element buffers [24][NE]
struct FomB {
    int n_inst;
    const InstFom* inst;
    long long NN, NE;
    const int2* eblk;         // element blocks: (instance, first element), eblock elements each
    int n_eblk, eblock;
    const int2* nblk;         // node blocks: (instance, first node), kNodeBlock nodes each
    int n_nblk;
    const int* nblk_off;      // [n_inst + 1] first node block of each instance
    const double* minv;
    const double* mass;       // lumped mass itself (implicit groups: the Newton system's M, no division)
    const uint8_t* clamp;
    const int* srow;
    double* u[2];
    double* v;
    double* a;
    void* f;                  // atomic accumulator [3][NN] (double, or float for FP32 force)
    void* fe;                 // element buffer [24][NE] (double, or float for FP32 force)
    double* su;
    double* sv;
    double* sa;
    double* pu;
    double* pv;
    double* hist;             // per instance [(nsub+1)][3 fields][3 comps][ns] at hist_off
    double* partial;          // criterion partial sums, 2 per node block
    double* us;               // predicted displacement divided by h [3][NN] (input of the FP64 / FP32 force)
    float2* u2;               // (hi, lo) float split of the predicted displacement / h [3][NN] (f32x2 and FP32 force)
    int material, fp32, scatter;
    int occ;                  // 1: FP64 gather force capped at 128 registers
    const int4* tblk;         // 8x4x4 element tiles: (instance, i0, j0, k0)
    int n_tblk;
    int tiled;                // 1: FP64 force by tiles (shared edge interpolation)
    // implicit Newmark (average acceleration) groups: Newton with a matrix-free CG per substep
    int implicit;
    double* ut;               // predictor [3][NN]
    double* cg_x;             // Newton increment [3][NN]
    double* cg_r;             // CG residual [3][NN]
    double* cg_p;             // CG direction [3][NN]
    double* cg_ap;            // tangent times direction [3][NN]
    double* ipart;            // partial sums, two per node block
    double* rn2;              // per instance: squared Newton residual
    double* r0;               // per instance: squared residual of the predictor
    double* rr;               // per instance: r . z of the current CG iterate (z = M^-1 r / c0)
    double* rrn;              // per instance: r . z after the update
    double* rr0;              // per instance: r . z at the start of the CG solve
    double* pap;              // per instance: p . A p
    double* cgtol2;           // per instance: squared relative CG tolerance of the current Newton step
    int* iloop;               // device-side loop counters: [0] Newton steps, [1] CG iterations
    unsigned int* iticket;    // per instance: last-block ticket of the fused CG reductions
    double* alpha;            // per instance: CG step length of the current iteration
    double* beta;             // per instance: CG direction update of the current iteration
    int* nact;                // per instance Newton state: 1 iterating, 0 converged, 2 failed
    int* cgact;               // per instance: CG still iterating
    long long* istat;         // per instance: Newton linear solves, CG iterations (since the last reset)
    double* lin;              // Neo-Hookean implicit groups: stored Newton linearisation [kLinPerGp][8][NE]
    float* linf;              // the same in FP32 (OSAM_FP64_TANGENT32; lin is then null)
    float* fe32;              // FP32 element buffer [24][NE] of the FP32 tangent action
    int df32;                 // 1: internal force in double-float arithmetic (element buffer of float2)
};

// one instance of a ROM slot
struct InstRom {
    int r, rs, nsdof, d, nq, nc, gx, gy;   // nc: cubic columns r(r+1)(r+2)/6 (0: quadratic ROM)
    long long O_off, PhiSt_off, kij_off, kijk_off, q_off, qrec_off, ghat_off, hist_off, partial_off;
};

struct RomB {
    int n_inst;
    const InstRom* inst;
    int gx_max, gy_max, rs_max, r_max;
    const double* O;          // packed operator rows [r][K | H | C | B | c] per instance (C: cubic ROMs)
    const double* PhiSt;      // Phi_S^T [rs][nsdof] per instance
    const short2* kij;        // compressed Kronecker index pairs per instance
    const short4* kijk;       // compressed Kronecker index triples per instance (cubic ROMs)
    double* q;                // [3][r] per instance: q, qd, qdd
    double* sq;
    double* pq;
    double* qrec;             // [(nsub+1)][3][r] per instance
    double* ghat;             // [(nsub+1)][rs] per instance
    double* hist;             // [(nsub+1)][3][nsdof] per instance
    double* partial;          // reduced-step partial sums [gx][r] per instance
    unsigned int* counter;    // [n_inst] last-block counters of the reduced step
    double* npart;            // criterion partial sums, 2 per instance
};

// one coupling (dst slot <- src slot) across instances; rows are concatenated over instances
struct CplB {
    int R;                    // total rows
    const int* rinst;         // instance of each row
    const int* row_first;     // [n_inst] first row of each instance
    const int* nrow;          // [n_inst] rows per instance
    const int* row;           // dst Schwarz row (local to the instance) of each row
    const int* dnode;         // [R][8] donor nodes, global index in the src group's node arrays
    const double* dw;         // [R][8] trilinear weights
    double* rec;              // FOM source: recorded trace, per instance [(nsub_src+1)][3][3][nrow]
    const long long* rec_off; // [n_inst]
    const double* Rt;         // ROM source: (Pi Phi_rows)^T, per instance [r][3 nrow]
    const long long* Rt_off;  // [n_inst]
    double* dst_hist;
    const long long* dst_hist_off;  // [n_inst]
    const int* dst_nd;        // [n_inst] dst Schwarz rows (FOM) or Schwarz dofs (ROM)
    int dst_rom;
};

// overlap traces folded into an internal-force launch as extra blocks at the end of its grid: the
// trace of substep j (u^j, v^j, a^j at the neighbours' Schwarz nodes) is taken while the force of
// substep j+1 runs, when u^j, v^j and a^j are still intact
constexpr int kMaxFusedTraces = 2;
struct TraceFuse {
    int n = 0;                // couplings (0: none)
    CplB c[kMaxFusedTraces];
    const double* u = nullptr;
    int slot = 0;
};

// per-instance controller state and criterion arguments
struct CtlB {
    int n_inst, n_fom, n_rom, ncpl, max_it;
    double tol_abs2, tol_rel2;
    const double* fom_partial[kMaxSlots];
    const int* fom_blk_off[kMaxSlots];
    const double* rom_npart[kMaxSlots];
    int* active;
    int* iters;
    int* status;
    double* cnum;
    double* cden;
    unsigned int* counter;
    int* any_active;
};

// ------------------------------------------------------------------------------------------------
// element level, set-up and I/O (fom_kernels.cu)
// ------------------------------------------------------------------------------------------------
int grid_for(long long n, int block);
cudaError_t launch_hex8_force(int material, bool fp32, int scatter, const ElemArgs& a, cudaStream_t s);
cudaError_t launch_lumped_minv(const Grid& g, double rho, double* minv, cudaStream_t s, double* mass = nullptr);
cudaError_t launch_donor(const Grid& src, const Grid& dst, const int* dst_nodes, int nrow, int* dnode, double* dw,
                         int* err, cudaStream_t s);
cudaError_t launch_aos_to_soa(const double* aos, double* soa, int nn, long long stride, cudaStream_t s);
cudaError_t launch_soa_to_aos(const double* soa, double* aos, int nn, long long stride, cudaStream_t s);
cudaError_t launch_cfl_modulus(const FomB& g, unsigned long long* out, int* bad, cudaStream_t s);
cudaError_t launch_zero_clamped(int nn, const uint8_t* clamp, double* u, double* v, long long stride, cudaStream_t s);

// ------------------------------------------------------------------------------------------------
// batched per-step kernels (step_kernels.cu); `active` masks instances that have converged
// ------------------------------------------------------------------------------------------------
// internal force of the predicted displacement held (divided by h) in g.us / g.u2
cudaError_t launch_force_b(const FomB& g, const int* active, int scatter, cudaStream_t s,
                           const TraceFuse* tr = nullptr);
cudaError_t launch_force_init_b(const FomB& g, const int* active, cudaStream_t s);  // FP64 gather of f(u[0]) into fe
cudaError_t launch_init_accel_b(const FomB& g, const int* active, cudaStream_t s);  // a = -M^-1 f from fe
cudaError_t launch_node_b(const FomB& g, const int* active, int scatter, int slot1, int slot2, int predict_only,
                          const double* ucur, double* unext, double dt, cudaStream_t s);
cudaError_t launch_saverest_fom_b(const FomB& g, const int* active, int restore, cudaStream_t s);
cudaError_t launch_norms_fom_b(const FomB& g, const int* active, double dt, cudaStream_t s);
cudaError_t launch_copy_u10_b(const FomB& g, const int* active, cudaStream_t s);
// double-float mode (force_df.cu)
cudaError_t launch_split_u2_b(const FomB& g, cudaStream_t s);
cudaError_t launch_force_df_b(const FomB& g, const int* active, const TraceFuse& tr, cudaStream_t s);
cudaError_t launch_node_df_b(const FomB& g, const int* active, int slot1, int slot2, int predict_only,
                             const double* ucur, double* unext, double dt, cudaStream_t s);
cudaError_t launch_trace_b(const CplB& c, const int* active, const FomB& src, const double* u, int slot,
                           cudaStream_t s);
// destination levels [slot0, slot0 + nslots) of nd from the source trace's levels 0..ns (temporal
// interpolant: linear between bracketing source levels, identity for ns == nd)
cudaError_t launch_publish_b(const CplB& c, const int* active, int slot0, int nslots, int ns, int nd, cudaStream_t s);
// zero-order hold into destination levels 0..nd and trace level 0
cudaError_t launch_zoh_fom_b(const CplB& c, const int* active, const FomB& src, int nd, cudaStream_t s);
cudaError_t launch_rom_record0_b(const RomB& r, const int* active, cudaStream_t s);
cudaError_t launch_rom_project_b(const RomB& r, const int* active, int slot0, int slot1, cudaStream_t s);
cudaError_t launch_rom_step_b(const RomB& r, const int* active, int slot, double dt, int rhs_only, cudaStream_t s);
// ROM source -> destination levels 1..nd (zoh: 0..nd from the current state) from ns source levels
cudaError_t launch_rom_reconstruct_b(const CplB& c, const int* active, const RomB& src, int zoh, int ns, int nd,
                                     cudaStream_t s);
cudaError_t launch_rom_norms_b(const RomB& r, const int* active, double dt, cudaStream_t s);
cudaError_t launch_saverest_rom_b(const RomB& r, const int* active, int restore, cudaStream_t s);
cudaError_t launch_reset_ctl(const CtlB& c, cudaStream_t s);
cudaError_t launch_controller(const CtlB& c, cudaGraphConditionalHandle h, int use_cond, cudaStream_t s);

// implicit Newmark, beta = 1/4, gamma = 1/2 (implicit_kernels.cu); `mask` = per-instance activity
cudaError_t launch_imp_predict_b(const FomB& g, const int* active, int slot1, double dt, cudaStream_t s);
cudaError_t launch_imp_residual_b(const FomB& g, const int* mask, double c0, cudaStream_t s);
// reduce the node-block partials per instance; mode 0: Newton residual (sets rn2, r0 on the first
// iteration (first < 0: the device-side Newton counter decides), rr, rr0, nact, cgact and the CG
// forcing tolerance), 3: |du|^2 <= tol2 |u|^2 after a Newton update (clears nact).  The CG inner
// products are reduced inside k_cg_ap_b / k_cg_step_b by each instance's last block.
cudaError_t launch_imp_reduce_b(const FomB& g, const int* mask, int mode, int first, double tol2, cudaStream_t s);
cudaError_t launch_tangent_b(const FomB& g, const int* mask, cudaStream_t s);
// Neo-Hookean implicit groups: Newton force that also stores the Gauss-point linearisation, and the
// tangent action that reads it
cudaError_t launch_force_lin_b(const FomB& g, const int* mask, cudaStream_t s);
cudaError_t launch_tangent_lin_b(const FomB& g, const int* mask, cudaStream_t s);
cudaError_t launch_cg_ap_b(const FomB& g, const int* mask, double c0, cudaStream_t s);
cudaError_t launch_cg_step_b(const FomB& g, const int* mask, double c0, double tol2, cudaStream_t s);
cudaError_t launch_cg_dir_b(const FomB& g, const int* mask, double c0, cudaStream_t s);
cudaError_t launch_imp_update_b(const FomB& g, const int* mask, cudaStream_t s);
cudaError_t launch_imp_finish_b(const FomB& g, const int* active, int slot1, double dt, double c0, cudaStream_t s);
cudaError_t launch_mask_copy(int n, const int* src, int* dst, cudaStream_t s);
// device-side loop control of the implicit solve (conditional WHILE nodes): which 0 Newton, 1 CG
cudaError_t launch_imp_loop_entry(const FomB& g, cudaGraphConditionalHandle h, int which, cudaStream_t s);
cudaError_t launch_imp_loop_cond(const FomB& g, cudaGraphConditionalHandle h, int which, int max_it, cudaStream_t s);

// ROM set-up and I/O (rom_kernels.cu)
cudaError_t launch_rom_basis_project(int nfree, int r, const double* Phi, const int* free_dof, const double* u_aos,
                                     const double* v_aos, double* q, cudaStream_t s);
cudaError_t launch_rom_full_field(int nn, int r, const double* Phi, const int* dof_free, const uint8_t* clamp,
                                  const int* srow, const double* hist_slot_field, const double* qv, double* out_aos,
                                  cudaStream_t s);
cudaError_t launch_build_Rt(int nrow, int r, const int* dnode_local, const double* dw, const int* dof_free,
                            const int* srow, const double* Phi, double* Rt, int* err, cudaStream_t s);

// dense helpers (fit)
// GEMM accounting of the fit (osam_fit_profile)
int gemm_profile(int enable, double* ms, double* flops, long long* launches);
cudaError_t launch_gemm_tn(int m, int n, int k, const double* A, int lda, const double* B, int ldb, double* C,
                           int ldc, double alpha, double beta, cudaStream_t s);
cudaError_t launch_gemm_nn(int m, int n, int k, const double* A, int lda, const double* B, int ldb, double* C,
                           int ldc, double alpha, double beta, cudaStream_t s);
cudaError_t launch_gemm_nt(int m, int n, int k, const double* A, int lda, const double* B, int ldb, double* C,
                           int ldc, double alpha, double beta, cudaStream_t s);
cudaError_t launch_kron_features(const double* Ubar, int r, int nsnap, double* D, int ldd, int col0,
                                 cudaStream_t s);
// compressed Kronecker cube (q_i q_j q_k)_{i<=j<=k} of every snapshot into columns col0.. of D
cudaError_t launch_kron3_features(const double* Ubar, int r, int nsnap, double* D, int ldd, int col0,
                                  cudaStream_t s);
// regularisation selection: nl candidate ROMs (packed rows [nl][r][d]) rolled out under frozen
// boundary data (D's boundary columns), error sums per candidate
cudaError_t launch_select_rollout(int nl, int r, int d, int nq, int nc, int rs, const double* O, const short2* kij,
                                  const short4* kijk, const double* D, const double* Y, const double* qd0, int ns,
                                  int k, double dt, double* phi, double* num, double* den, cudaStream_t s);

// adjoint (adjoint_kernels.cu)
cudaError_t launch_hex8_vjp(int material, int scatter, const ElemArgs& a, const double* ybar, int ysn, long long ysc,
                            double* lam_bar, double* mu_bar, int acc, cudaStream_t s);
cudaError_t launch_adjoint_pre(int nn, double dt, const uint8_t* clamp, const double* minv, const double* vb, double* ab,
                               double* y, cudaStream_t s);
cudaError_t launch_adjoint_post(int nx, int ny, int nz, double dt, const uint8_t* clamp, const double* fe, double* ub,
                                double* vb, double* ab, cudaStream_t s);

// message returned by osam_last_error(NULL) on the calling thread
void set_thread_error(const std::string& msg);

}  // namespace osam
