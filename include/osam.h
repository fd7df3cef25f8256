/*
 * osam.h -- C ABI of libosam, the GB300 (sm_103a) implementation of one controller step of the
 * overlapping Schwarz alternating method (O-SAM) coupling hex8 full order models (FOMs) and
 * quadratic operator-inference (OpInf) reduced order models (ROMs) for 3D solid dynamics
 * (arXiv 2511.20687).
 *
 * Conventions used by every entry point
 *   - Subdomains are structured boxes of nx*ny*nz cubic hex8 elements of edge h with origin at the
 *     minimum corner.  Node (i,j,k) has index i + (nx+1)*(j + (ny+1)*k); element (i,j,k) has index
 *     i + nx*(j + ny*k).
 *   - Nodal fields passed across the ABI are interleaved [node][3] float64 arrays.
 *   - Per-node Dirichlet masks (uint8) have bit c set when displacement component c is clamped to 0.
 *   - Every pointer argument may be host memory (pageable or pinned) or device memory of the
 *     context's GPU unless stated otherwise; the library copies what it needs.  The caller owns every
 *     pointer it passes; the library never frees caller memory, never prints and never exits.
 *   - Return values are osam_status codes; negative values are errors, with a message available
 *     from osam_last_error().  OSAM_MAXITER is not an error: the controller step was committed after
 *     max_iters Schwarz iterations, as the paper continues after hitting its iteration cap (Sec. 5.4).
 *   - Calls are stream ordered on the context's stream and return after the work they describe has
 *     completed unless stated otherwise.
 *   - There is no CPU fallback: every step runs in the library's CUDA kernels and an error is
 *     returned when no usable sm_103a device is present.
 */
#ifndef OSAM_H
#define OSAM_H

#include <stdint.h>

#if defined(__GNUC__)
#define OSAM_API __attribute__((visibility("default")))
#else
#define OSAM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    OSAM_OK = 0,
    OSAM_MAXITER = 1,      /* non-fatal: controller step committed at the iteration cap */
    OSAM_EINVAL = -1,      /* invalid argument or inconsistent description */
    OSAM_ECFL = -2,        /* explicit time step above the stability limit */
    OSAM_ENONFINITE = -3,  /* NaN or Inf in the coupled state (cf. the non-finite ROM penalty, Alg. 3) */
    OSAM_EDONOR = -4,      /* a Schwarz node has no donor element in its source subdomain */
    OSAM_ECUDA = -5,       /* CUDA runtime error, or no usable device */
    OSAM_ETIMEOUT = -6,    /* a bounded device-side wait gave up */
    OSAM_ENOMEM = -7       /* device allocation failed */
} osam_status;

enum { OSAM_FOM = 0, OSAM_ROM = 1 };
enum { OSAM_LINEAR_ELASTIC = 0, OSAM_NEO_HOOKEAN = 1, OSAM_SAINT_VENANT_KIRCHHOFF = 2 };
/* FOM time integrator: explicit Newmark (beta = 0, gamma = 1/2, central difference) or implicit
 * Newmark (beta = 1/4, gamma = 1/2, average acceleration) */
enum { OSAM_EXPLICIT = 0, OSAM_IMPLICIT = 1 };
enum { OSAM_MULTIPLICATIVE = 0, OSAM_ADDITIVE = 1 };
/* OSAM_FP64: native FP64 everywhere.  OSAM_FP32_FORCE: internal force in FP32 (checked to 1e-5).
 * OSAM_F32X2_FORCE: internal force in double-float arithmetic (pairs of FP32 values, ~48-bit
 * significands) on the FP32 pipes, state and time integration in FP64 (checked to 1e-9 like FP64);
 * uses the deterministic gather scatter.  OSAM_FP64_TANGENT32: OSAM_FP64, except that the Newton
 * tangent of implicit Neo-Hookean subdomains (its stored Gauss-point linearisation, its action on
 * the conjugate-gradient direction and the element contributions of that action) is in FP32; the
 * Newton residual and its test, the CG vectors and reductions stay FP64, so a converged step meets the
 * same FP64 residual test as OSAM_FP64 (inexact Newton with a lower-precision inner solve; each CG
 * solve stops at a relative tolerance of at least 1e-6).  Explicit subdomains run as OSAM_FP64. */
enum { OSAM_FP64 = 0, OSAM_FP32_FORCE = 1, OSAM_F32X2_FORCE = 2, OSAM_FP64_TANGENT32 = 3 };
/* element-to-node scatter of the internal force: FP64 atomics, or a deterministic two-pass
 * element-buffer / node-gather scheme; GATHER_LOWREG is the gather scheme with the FP64 force kernel
 * compiled for at most 128 registers per thread (more resident warps, a few spilled values);
 * GATHER_TILED the gather scheme with the FP64 force evaluated by 8x4x4 element tiles that share
 * their edge interpolation (same results bit for bit), GATHER_TILED_LOWREG the tiled kernel capped at
 * 128 registers (4 instead of 3 resident tiles per SM); the FP32 variants ignore these.  AUTO times
 * the candidates at initialisation and keeps the fastest */
enum {
    OSAM_SCATTER_AUTO = 0,
    OSAM_SCATTER_ATOMIC = 1,
    OSAM_SCATTER_GATHER = 2,
    OSAM_SCATTER_GATHER_LOWREG = 3,
    OSAM_SCATTER_GATHER_TILED = 4,
    OSAM_SCATTER_GATHER_TILED_LOWREG = 5   /* the tiled FP64 force capped at 128 registers (4 tiles per SM) */
};

typedef struct osam_ctx osam_ctx;

/* One subdomain (Sec. 4, Eq. dynamic_elasticity_sam_bcs).
 * FOM: hex8 isoparametric FE (Sec. 2, Eq. matrix_vector_form) with 2x2x2 Gauss quadrature,
 *   row-sum lumped mass, explicit Newmark beta=0 gamma=1/2 (Sec. 5 setup) or implicit Newmark
 *   beta=1/4 gamma=1/2 (Sec. 4.1, `integrator`), material of Appendix A.1
 *   (linear elastic) or A.3 (Neo-Hookean, deviatoric coefficient 1/3 from its energy).
 * ROM: quadratic OpInf model of Eq. opinf_model_schwarz in solved form
 *   qdd = K q + H kron_c(q) + B ghat + c,  ghat = Phi_S^T s  (Sec. 4.2.1, boundary POD),
 *   kron_c(q) = (q_i q_j)_{i<=j} in row-major upper-triangle order; the ROM's free dofs are all dofs
 *   of its mesh that are neither clamped nor on a Schwarz node (increasing dof id 3*node+c), its
 *   Schwarz dofs are the 3 components of every Schwarz node (increasing node order). */
typedef struct {
    int kind;                 /* OSAM_FOM or OSAM_ROM */
    int nx, ny, nz;           /* elements per direction (>= 1) */
    double h;                 /* element edge (> 0) */
    double origin[3];
    /* FOM material */
    int material;             /* OSAM_LINEAR_ELASTIC, OSAM_NEO_HOOKEAN or OSAM_SAINT_VENANT_KIRCHHOFF (A.2:
                               * E = 1/2 (F^T F - I), S = lambda tr(E) I + 2 mu E, P = F S) */
    double lambda, mu, rho;   /* Lame parameters and density (kappa = lambda + 2/3 mu for NH) */
    const double* lambda_e;   /* optional per-element Lame parameters [nx*ny*nz], NULL = uniform */
    const double* mu_e;
    const uint8_t* dirichlet; /* per-node clamp mask [nodes] or NULL */
    const double* u0;         /* initial displacement [nodes][3] (required) */
    const double* v0;         /* initial velocity [nodes][3] or NULL (zero) */
    /* ROM operators (kind == OSAM_ROM), all row-major float64 */
    int r, r_s;               /* reduced dimension (1..256; 1..128 with a cubic operator C) and boundary
                               * reduced dimension (>= 0; 0 = no boundary input); else OSAM_EINVAL */
    const double* Phi;        /* [n_free][r] orthonormal POD basis */
    const double* Phi_S;      /* [3*n_schwarz_nodes][r_s] boundary POD basis */
    const double* K;          /* [r][r] */
    const double* H;          /* [r][r(r+1)/2] */
    const double* B;          /* [r][r_s] */
    const double* c;          /* [r] */
    /* FOM integrator (OSAM_EXPLICIT or OSAM_IMPLICIT; ignored for ROMs).  An implicit FOM solves
     * M (u - u~) / (beta dt^2) + f_int(u) = 0 on its free dofs each substep (u~ the Newmark predictor)
     * by Newton's method, |R| <= 1e-12 |R(u~)| within 25 iterations, each Newton system by conjugate
     * gradients with the exact tangent applied matrix-free (Appendix A tangents).  No stability
     * limit applies to it.  Implicit FOMs need OSAM_FP64 and run host-driven (no CUDA graph); a Newton
     * solve that fails leaves a non-finite state, reported as OSAM_ENONFINITE. */
    int integrator;
    /* substeps of this subdomain per controller step (Sec. 4.1: n_i, Delta t_i = dt n_substeps / n_i of
     * the problem; 0 = the problem's n_substeps).  Schwarz data between subdomains with different
     * counts go through the temporal interpolant Xi: linear in time between the two source levels
     * that bracket each destination level (identity for equal counts). */
    int n_substeps;
    /* cubic OpInf (COpInf, Eq. opinf_rom with all terms): qdd += C kron3_c(q), kron3_c(q) =
     * (q_i q_j q_k)_{i<=j<=k} in lexicographic order; [r][r(r+1)(r+2)/6] row-major, or NULL for the
     * quadratic model; r <= 128 with it */
    const double* C;
} osam_subdomain_desc;

/* Dirichlet transfer from subdomain src to the Schwarz boundary nodes of dst (Sec. 4.1): the data
 * on node n of dst is the trilinear interpolant (pointwise projector Pi) of src's solution at the
 * position of n, in the lowest-index src element containing it (local coordinates within 1e-9 of
 * +-1 are snapped to +-1).  nodes: uint8 [dst nodes], nonzero = Schwarz node fed by src. */
typedef struct {
    int dst, src;
    const uint8_t* nodes;
} osam_coupling_desc;

typedef struct {
    int n_subdomains;
    const osam_subdomain_desc* subdomains;
    int n_couplings;
    const osam_coupling_desc* couplings;
    double dt;                /* time step of every subdomain with the default substep count */
    int n_substeps;           /* substeps per controller step I_k (its length is dt n_substeps) */
    double tol_abs, tol_rel;  /* delta_abs, delta_rel of Eq. conv_criterion (0 disables a test) */
    int max_iters;            /* Schwarz iteration cap per controller step */
    int precision;            /* OSAM_FP64 or OSAM_FP32_FORCE (internal force in FP32) */
    int scatter;              /* OSAM_SCATTER_* */
    void* stream;             /* cudaStream_t to run on, or NULL for a library-owned stream */
    int device;               /* CUDA device ordinal */
    /* OSAM_MULTIPLICATIVE (Algorithm 1: subdomains in index order, each from the data its
     * predecessors published in the same iteration) or OSAM_ADDITIVE (Remark additive_sam: every
     * subdomain from the previous iteration's data, all subdomains advanced concurrently on their own
     * streams, then every transfer) */
    int schwarz;
} osam_problem_desc;

typedef struct {
    int status;               /* OSAM_OK or OSAM_MAXITER (errors are returned, not reported here) */
    int iterations;           /* Schwarz iterations performed */
    double cnum, cden;        /* numerator / denominator sums of Eq. conv_criterion at the last iteration */
    long long element_updates;/* FOM elements x substeps executed in this step */
    double elapsed_ms;        /* device time of the step (CUDA events on the context stream) */
} osam_step_report;

/* Build the coupled problem on the device: meshes, lumped masses, node sets, donor elements and
 * trilinear weights of every Schwarz node (Pi, Sec. 4.1), ROM operators, initial accelerations.
 * Initial boundary data come from the sources' initial states.  Allocates all device memory the
 * context will use.  *out receives the context (NULL on error; the error text is then available from
 * osam_last_error(NULL) on the calling thread). */
OSAM_API int schwarz_init(const osam_problem_desc* desc, osam_ctx** out);

/* Advance subdomain `sub` over the current controller interval (n_substeps steps) from its current
 * state, with Dirichlet data from its input boundary history (Eq. schwarz_discrete / Eq.
 * schwarz_opinf_discrete), and record its trace at every Schwarz node it feeds.  The step count is the
 * subdomain's own substep count from its description (osam_subdomain_desc.n_substeps, else the
 * problem's), not an argument: the boundary history, the temporal interpolant and the criterion are
 * all laid out for that count when the context is built, so a different count per call would have no
 * matching boundary data. */
OSAM_API int subdomain_advance(osam_ctx* ctx, int sub);

/* Publish src's recorded trace of the current interval into dst's input boundary history -- the
 * Schwarz Dirichlet data of Eq. schwarz_discrete / Eq. schwarz_opinf_discrete (Sec. 4.1): the
 * projection Pi at dst's Schwarz nodes, taken onto dst's levels by the temporal interpolant Xi.
 * FOM->FOM copy; FOM->ROM the ROM's boundary snapshot rows; ROM->any Pi Phi q at every substep. */
OSAM_API int transfer_overlap(osam_ctx* ctx, int src, int dst);

/* Start a controller interval of Algorithm 1: save every state at t_{k-1} and fill every input
 * boundary history with the zero-order hold of its source's state at t_{k-1} (initial guess of
 * iteration 1). */
OSAM_API int osam_begin_interval(osam_ctx* ctx);

/* Return every subdomain to the state saved by osam_begin_interval (start of a new Schwarz iteration
 * of Algorithm 1). */
OSAM_API int osam_restore_interval(osam_ctx* ctx);

/* Sums of Eq. conv_criterion between the current end states and those of the previous call:
 * cnum = sum_i ||du_i + dt dv_i||^2, cden = sum_i ||u_i + dt v_i||^2 over free dofs (ROM: over q, qd,
 * equal to the full-space norms for an orthonormal Phi).  Remembers the current states. */
OSAM_API int osam_criterion(osam_ctx* ctx, double* cnum, double* cden);

/* One controller step (Algorithm 1): begin interval; for n = 1..max_iters: restore (n > 1),
 * advance every subdomain in index order publishing its traces, criterion; converged when n >= 2 and
 * cnum < tol_abs^2 or cnum < tol_rel^2 cden.  rep may be NULL. */
OSAM_API int schwarz_step(osam_ctx* ctx, osam_step_report* rep);

/* ------------------------------------------------------------------------------------------------
 * Batches: one context advancing n_instances independent instances of the same coupled problem
 * (same subdomain kinds and Neo-Hookean / linear-elastic choice per subdomain, same couplings, dt,
 * n_substeps, tolerances, max_iters and precision; meshes, materials, initial data and ROM operators
 * may differ per instance).  Every per-step kernel advances all instances in one launch; an instance
 * that meets the criterion stops iterating (its state is frozen) while the others continue, so each
 * instance follows exactly its own single-instance iteration sequence.  schwarz_init is a batch of
 * one.  The instance index of the functions below is 0-based; functions without it act on instance 0.
 * Batching has no counterpart in the paper: each instance runs Algorithm 1 unchanged.
 * ------------------------------------------------------------------------------------------------ */
OSAM_API int osam_batch_init(int n_instances, const osam_problem_desc* descs, osam_ctx** out);
/* One controller step of every instance; per_instance[n_instances] (or NULL) receives each instance's
 * report, total (or NULL) the aggregate (iterations = max, element_updates = sum, status = worst). */
OSAM_API int osam_batch_step(osam_ctx* ctx, osam_step_report* per_instance, osam_step_report* total);
OSAM_API int osam_num_instances(osam_ctx* ctx);
OSAM_API int osam_instance_get_state(osam_ctx* ctx, int inst, int sub, double* u, double* v, double* a);
OSAM_API int osam_instance_set_state(osam_ctx* ctx, int inst, int sub, const double* u, const double* v, const double* a);
OSAM_API int osam_instance_get_reduced_state(osam_ctx* ctx, int inst, int sub, double* q, double* qd, double* qdd);
OSAM_API int osam_instance_set_reduced_state(osam_ctx* ctx, int inst, int sub, const double* q, const double* qd,
                                    const double* qdd);
OSAM_API int osam_instance_sizes(osam_ctx* ctx, int inst, int sub, int* n_nodes, int* n_elements, int* n_free,
                        int* n_schwarz_nodes);
/* Controller-step execution: enable = 1 (default) records the whole step once as a CUDA graph -- save,
 * zero-order hold, then a while node whose body is one Schwarz iteration of every instance and whose
 * condition is set on the device by the convergence kernel -- and replays it with one host
 * synchronisation per step; enable = 0 drives the iterations from the host (one synchronisation per
 * iteration).  Kernel-level profiling (osam_profile) always uses the host-driven path. */
OSAM_API int osam_set_graph(osam_ctx* ctx, int enable);
/* Autotuned launch configuration of the force kernel: scatter mode, element block size, register
 * cap (0: natural register count; 128: the FP64 gather kernel compiled for at most 128 registers per
 * thread) and tiling (1: the FP64 force by 8x4x4 element tiles).  Any pointer may be NULL. */
OSAM_API int osam_tuning(osam_ctx* ctx, int* scatter, int* element_block, int* register_cap, int* tiled);

/* Copy a subdomain's nodal state (u, v, a of Eq. schwarz_discrete at the end of the last committed
 * interval) out / in ([nodes][3] each, any pointer may be NULL).  For a ROM the
 * output is the reconstructed field: Phi q on free dofs, boundary data on Schwarz dofs, 0 on clamped
 * dofs; osam_set_state on a ROM projects u, v onto the basis (q = Phi^T u) and recomputes qdd. */
OSAM_API int osam_get_state(osam_ctx* ctx, int sub, double* u, double* v, double* a);
OSAM_API int osam_set_state(osam_ctx* ctx, int sub, const double* u, const double* v, const double* a);
/* Reduced state (q, qd, qdd of Eq. schwarz_opinf_discrete) of a ROM subdomain ([r] each). */
OSAM_API int osam_get_reduced_state(osam_ctx* ctx, int sub, double* q, double* qd, double* qdd);
OSAM_API int osam_set_reduced_state(osam_ctx* ctx, int sub, const double* q, const double* qd, const double* qdd);
/* Sizes of subdomain `sub` (any output may be NULL). */
OSAM_API int osam_sizes(osam_ctx* ctx, int sub, int* n_nodes, int* n_elements, int* n_free, int* n_schwarz_nodes);
/* Kernel-level accounting for measurement: with enable = 1, every internal-force launch of
 * schwarz_step / subdomain_advance is bracketed by CUDA events on the context stream; the counters
 * (force time, force launches, elements processed by them, and all kernel launches issued by the
 * controller) restart at zero on every osam_profile call. */
OSAM_API int osam_profile(osam_ctx* ctx, int enable);
OSAM_API int osam_profile_read(osam_ctx* ctx, double* force_ms, long long* force_launches, long long* force_elements,
                      long long* kernel_launches);
/* Accounting of the implicit subdomains since the last osam_profile call: time of the tangent-action
 * launches (CUDA events around each, recorded only while profiling is enabled) and their count,
 * elements whose tangent action was applied (CG iterations x elements, per instance), Newton linear
 * solves and CG iterations summed over instances and implicit subdomains.  Any output may be NULL. */
OSAM_API int osam_implicit_profile(osam_ctx* ctx, double* tangent_ms, long long* tangent_launches,
                                   long long* tangent_elements, long long* newton_steps, long long* cg_iterations);
/* FP64 fused multiply-add throughput of device `device` in GFLOP/s (2 flops per FMA), measured by a
 * register-resident FMA loop over 8 blocks per SM (best of five launches); the ALU roofline of the
 * FP64 element kernels. */
OSAM_API int osam_fp64_peak(int device, double* gflops);
/* FP64 throughput probe: `repeats` launches (1..1000) of about 20 ms each on device `device`, each
 * reported as TFLOP/s in tflops[r] and, if ms is not NULL, its CUDA-event duration in ms[r].
 * kind 0: FMA on the FP64 pipe (8 register chains per thread); kind 1: FP64 tensor-core MMA
 * (mma.sync m8n8k4, 4 accumulator chains per warp); kind 2: both interleaved in the same warps
 * (total flops), which shows whether the two share one unit.  Synchronous; allocates a small
 * output buffer.  Bad arguments -> OSAM_EINVAL. */
OSAM_API int osam_fp64_probe(int device, int kind, int repeats, double* tflops, double* ms);
/* FP64 issue probe: one block of `warps` warps (1..32), `lanes` active lanes each (1..32), running
 * 8 independent FMA chains per thread alone on one SM of device `device`; *ns_per_instruction = the
 * time per FP64 warp-instruction of one warp (best of three launches of ~160,000 instructions per
 * warp).  With few warps per SM sub-partition this is the latency floor of an element kernel on a
 * small mesh.  Synchronous; allocates a small output buffer.  Bad arguments -> OSAM_EINVAL. */
OSAM_API int osam_fp64_issue_probe(int device, int warps, int lanes, double* ns_per_instruction);
/* The scatter mode in use (OSAM_SCATTER_ATOMIC / GATHER) after any autotuning. */
OSAM_API int osam_scatter_mode(osam_ctx* ctx);
/* Free every resource of ctx (library-owned memory, streams, graphs); caller memory is untouched.
 * NULL is a no-op. */
OSAM_API void osam_destroy(osam_ctx* ctx);
/* Message of the last error on ctx, or of the calling thread's last failed schwarz_init if ctx is NULL. */
OSAM_API const char* osam_last_error(const osam_ctx* ctx);

/* ------------------------------------------------------------------------------------------------
 * Element-level operators on device arrays (device pointers only, [nodes][3] layout, stream ordered,
 * asynchronous).  Internal force f = sum_e sum_gp w detJ P(F) grad N (Sec. 2, Eq. weak_form with
 * the materials of Appendix A) and its vector-Jacobian product
 *   ubar = (df/du)^T ybar,  lambda_bar[e] = ybar . df/dlambda_e,  mu_bar[e] = ybar . df/dmu_e.
 * lambda_e / mu_e: per-element device arrays or NULL for the uniform lambda / mu.
 * Meshes whose element count or 3 x node count exceeds INT_MAX -> OSAM_EINVAL; every OSAM_EINVAL
 * leaves its reason in osam_last_error(NULL).
 * ------------------------------------------------------------------------------------------------ */
OSAM_API int osam_hex8_force(int nx, int ny, int nz, double h, int material, double lambda, double mu,
                    const double* lambda_e, const double* mu_e, const double* u, double* f, void* stream);
OSAM_API int osam_hex8_force_vjp(int nx, int ny, int nz, double h, int material, double lambda, double mu,
                        const double* lambda_e, const double* mu_e, const double* u, const double* ybar,
                        double* ubar, double* lambda_bar, double* mu_bar, void* stream);

/* Internal force for callers that may not allocate device memory (the paper has no counterpart):
 * an application that freezes its GPU memory budget after start-up and forbids cudaMalloc / cudaFree
 * (they can synchronise the device and fragment a pool the application manages), code running inside
 * another allocator's hooks, or a thread that must never block on cudaFree's implicit
 * synchronisation.  Same inputs, layout and result as osam_hex8_force (device pointers, [nodes][3]),
 * computed with the deterministic element-buffer scatter; the buffer is a static device array of
 * 24 * OSAM_NOALLOC_MAX_ELEMENTS doubles (6 MiB).  A dimension or an element count above
 * OSAM_NOALLOC_MAX_ELEMENTS -> OSAM_EINVAL (message in osam_last_error(NULL)).
 * Set-up: the first call on a device, with that device current, does a one-time set-up on `stream`
 * and waits for it: it looks up the array's device address and runs each kernel of this entry point
 * once on a one-element mesh.  The CUDA runtime loads the array and the kernels' code lazily, so this
 * first call is the one that makes the device take the 6 MiB (and the code); make it during start-up
 * (a 1x1x1 mesh is enough), before the memory budget is frozen and before any stream capture.  Later
 * calls on that device call no allocator and do not synchronise.  The device then holds the array
 * until the process exits.
 * Every call shares the one buffer and overwrites it entirely (nothing in it needs to start at zero):
 * calls whose kernels overlap on the GPU (different streams, or different host threads on one device)
 * race and must be serialised by the caller.  Asynchronous on `stream` after the set-up. */
#define OSAM_NOALLOC_MAX_ELEMENTS 32768
OSAM_API int osam_hex8_force_noalloc(int nx, int ny, int nz, double h, int material, double lambda, double mu,
                            const double* lambda_e, const double* mu_e, const double* u, double* f, void* stream);

/* ------------------------------------------------------------------------------------------------
 * Offline OpInf (Sec. 3 and Sec. 4.2.1, Eq. opinf_schwarz_inference) on the GPU:
 *   POD of the free-dof displacement snapshots U (thin SVD by the method of snapshots, Eq.
 *   pod_cutoff), boundary POD of the Schwarz snapshots S with the smallest r_s whose energy
 *   E_r (Eq. pod_energy) reaches energy_s (capped at r_s_max; r_s > 0 in the input fixes it),
 *   projection Ubar = Phi^T U, Abar = Phi^T A, Ghat = Phi_S^T S, and the Tikhonov regression
 *   min ||D O - Abar^T||^2 + lambda ||O||^2, D = [Ubar^T, kron_c(Ubar)^T, (kron3_c(Ubar)^T,) Ghat^T, 1]
 *   (one scalar lambda for every block; the dual form D^T (D D^T + lambda I)^-1 Abar^T is used when
 *   D has more columns than rows).  Snapshot matrices are [n_snap][n_dof] (one snapshot per row).
 * ------------------------------------------------------------------------------------------------ */
typedef struct {
    int n_dof, n_snap, n_sdof;  /* each below 2^31 - 64 (else OSAM_EINVAL) */
    const double* U;          /* [n_snap][n_dof] displacement snapshots (free dofs) */
    const double* A;          /* [n_snap][n_dof] acceleration snapshots */
    const double* S;          /* [n_snap][n_sdof] Schwarz boundary displacement snapshots */
    int r;                    /* POD rank of U */
    int r_s;                  /* boundary rank, or 0 to select it by energy */
    double energy_s;          /* energy threshold for r_s (e.g. 1 - 1e-6) */
    int r_s_max;
    double lambda;
    int quadratic;            /* 1: quadratic OpInf, 0: linear (H = 0) */
    void* stream;
    int device;
    int cubic;                /* 1: cubic OpInf (COpInf): the block kron3_c(Ubar)^T after the quadratic one,
                               * operator C [r][r(r+1)(r+2)/6] (implies the quadratic block); r <= 128 */
} osam_fit_input;

typedef struct {
    double* Phi;              /* [n_dof][r] */
    double* Phi_S;            /* [n_sdof][r_s_max]; the first r_s columns are meaningful */
    double* K;                /* [r][r] */
    double* H;                /* [r][r(r+1)/2] */
    double* B;                /* [r][r_s_max]; the first r_s columns are meaningful */
    double* c;                /* [r] */
    double* sigma;            /* [n_snap] singular values of U, or NULL */
    double* sigma_s;          /* [n_snap] singular values of S, or NULL */
    int r_s;                  /* selected boundary rank */
    double* C;                /* [r][r(r+1)(r+2)/6] cubic operator (cubic fits), or NULL */
} osam_fit_output;

/* The regularisation lambda is a field of osam_fit_input (next to the other fit settings it goes with,
 * e.g. the same input serves opinf_select, which ignores it and scans its candidates) rather than a
 * separate argument. */
OSAM_API int opinf_fit(const osam_fit_input* in, osam_fit_output* out);

/* Schwarz-aware regularisation selection (Sec. 4.2.4, Algorithm 3): for every candidate lambda the
 * operators are fitted as by opinf_fit (in->lambda is ignored) and the ROM is advanced alone from
 * the training initial state (q0 = Phi^T u_0, qd0 = Phi^T v_0, qdd0 = Phi^T a_0, u_0 and a_0 the first
 * rows of U and A) by explicit central differences with step dt, its Schwarz boundary data frozen to
 * the training columns Ghat = Phi_S^T S; consecutive snapshot rows are `substeps` steps apart and the
 * boundary vector is interpolated linearly in time between them (substeps = 1: the stored column of
 * the new time level).  errors[l] = ||Q_l - Ubar||_F / ||Ubar||_F over the snapshot times
 * (Eq. schwarz_regularization_error), HUGE_VAL for a non-finite rollout; *best = the minimiser, whose
 * operators are written to out.  OSAM_ENONFINITE if every rollout is non-finite.  r <= 128. */
typedef struct {
    const double* lambdas;    /* [n_lambda] candidates (>= 0), e.g. 11 log-spaced values 1e-10 .. 1 */
    int n_lambda;             /* 1 .. 64 */
    const double* v0;         /* [n_dof] velocity of the first snapshot on the free dofs, or NULL (zero) */
    double dt;                /* rollout step (the ROM's online step) */
    int substeps;             /* steps between consecutive snapshot rows (>= 1) */
} osam_select_input;
OSAM_API int opinf_select(const osam_fit_input* in, const osam_select_input* sel, double* errors, int* best,
                          osam_fit_output* out);
/* Message of the calling thread's last failed opinf_fit / opinf_select. */
OSAM_API const char* osam_fit_last_error(void);
/* Accounting of the fit's device contractions on the calling host thread (a measurement hook; the
 * paper has no counterpart).  enable = 1 resets the counters and turns it on: every GEMM of a later
 * opinf_fit / opinf_select on this thread is bracketed by CUDA events and waited for (slower fits).
 * enable = 0 turns it off.  Either call returns, through the non-NULL pointers, the event time in ms,
 * the flops (2 m n k per product) and the number of GEMMs since the last reset. */
OSAM_API int osam_fit_profile(int enable, double* gemm_ms, double* gemm_flops, long long* gemm_launches);

/* ------------------------------------------------------------------------------------------------
 * Adjoint of the explicit single-domain rollout (gradients through the central-difference scheme
 * of Sec. 5 with the hex8 force and its VJP): J = w . u_T after n_steps steps from (u0, v0),
 * gradients w.r.t. u0, v0 and the per-element Lame parameters.  The forward pass stores (u, v, a)
 * every checkpoint_every steps; the reverse sweep recomputes each segment.  Outputs are host or
 * device pointers ([nodes][3] or [elements]); any may be NULL.
 * ------------------------------------------------------------------------------------------------ */
typedef struct {
    int nx, ny, nz;
    double h;
    int material;
    const double* lambda_e;   /* [elements] (required) */
    const double* mu_e;       /* [elements] (required) */
    double rho;
    const uint8_t* dirichlet; /* per-node clamp mask or NULL */
    const double* u0;         /* [nodes][3] */
    const double* v0;         /* [nodes][3] or NULL */
    double dt;
    int n_steps;
    int checkpoint_every;
    const double* w;          /* [nodes][3] weights of J */
    void* stream;
    int device;
} osam_adjoint_desc;

typedef struct {
    double J;
    double* grad_u0;          /* [nodes][3] */
    double* grad_v0;          /* [nodes][3] */
    double* grad_lambda;      /* [elements] */
    double* grad_mu;          /* [elements] */
    double elapsed_ms;        /* device time of forward + reverse */
} osam_adjoint_out;

OSAM_API int osam_adjoint(const osam_adjoint_desc* d, osam_adjoint_out* out);

#ifdef __cplusplus
}
#endif

#endif /* OSAM_H */
