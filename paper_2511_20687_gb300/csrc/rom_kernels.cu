// OpInf ROM subdomain kernels (Sec. 4.2, Eq. schwarz_opinf_discrete in solved explicit form):
//   boundary projection    ghat^j = Phi_S^T s^j                         (boundary POD, Sec. 4.2.1)
//   reduced step           qdd' = K q + H kron_c(q) + B ghat + c, explicit central difference
//   reconstruction         s_dst^j = (Pi Phi_rows) q^j at a neighbour's Schwarz nodes
//   criterion sums over (q, qd), basis projection q = Phi^T u, full-field reconstruction,
// and the dense FP64 products of the offline fit.
#include <cuda_runtime.h>

#include <cstdint>

#include "osam_internal.h"

namespace osam {

namespace {

constexpr int kRomBlock = 128;   // columns per block of the reduced step
constexpr int kRomRows = 8;      // rows per block of the reduced step
constexpr int kMaxR = 256;

__device__ __forceinline__ double block_sum(double x) {
    __shared__ double s[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    const int w = threadIdx.x / 32, l = threadIdx.x % 32;
    __syncthreads();
    if (l == 0) s[w] = x;
    __syncthreads();
    const int nw = (blockDim.x + 31) / 32;
    if (w == 0) {
        x = l < nw ? s[l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    }
    return x;  // valid in thread 0
}

// ghat[slot][k] = sum_m PhiSt[k][m] * hist[slot][field 0][m]; one block per (slot, k)
__global__ void k_rom_project(const double* PhiSt, const double* hist, double* ghat, int rs, int nsdof, int slot0) {
    const int k = blockIdx.x;
    const int slot = slot0 + blockIdx.y;
    const double* s = hist + (long long)slot * 3 * nsdof;
    const double* p = PhiSt + (long long)k * nsdof;
    double acc = 0.0;
    for (int m = threadIdx.x; m < nsdof; m += blockDim.x) acc = fma(p[m], s[m], acc);
    acc = block_sum(acc);
    if (threadIdx.x == 0) ghat[(long long)slot * rs + k] = acc;
}

struct RomStepArgs {
    int r, d, nq, rs;
    const double* O;
    const short2* kij;
    double* q;              // [3][r]: q, qd, qdd
    const double* ghat;     // [rs] of slot j+1
    double dt;
    double* partial;        // [gx][r]
    unsigned int* counter;
    double* qrec;           // [3][r] of slot j+1, or null
    int rhs_only;           // 1: qdd = rhs(q) without time stepping
};

// Column-split GEMV of the packed operator with the feature vector phi = [q, kron_c(q), ghat, 1]
// at the predicted q, then the last block to finish reduces the partial sums in fixed order
// (deterministic) and applies the corrector.
__global__ void __launch_bounds__(kRomBlock) k_rom_step(const RomStepArgs a) {
    __shared__ double qp[kMaxR];
    __shared__ double red[kRomBlock / 32][kRomRows];
    __shared__ bool last_block;
    const int tid = threadIdx.x;
    const double dt = a.dt;
    for (int t = tid; t < a.r; t += blockDim.x) {
        const double q = a.q[t];
        qp[t] = a.rhs_only ? q : fma(0.5 * dt * dt, a.q[2 * a.r + t], fma(dt, a.q[a.r + t], q));
    }
    __syncthreads();
    const int col = blockIdx.x * kRomBlock + tid;
    double phi = 0.0;
    if (col < a.r) phi = qp[col];
    else if (col < a.r + a.nq) { const short2 ij = a.kij[col - a.r]; phi = qp[ij.x] * qp[ij.y]; }
    else if (col < a.r + a.nq + a.rs) phi = a.ghat[col - a.r - a.nq];
    else if (col == a.d - 1) phi = 1.0;
    double part[kRomRows];
#pragma unroll
    for (int rr = 0; rr < kRomRows; ++rr) {
        const int row = blockIdx.y * kRomRows + rr;
        part[rr] = (row < a.r && col < a.d) ? a.O[(long long)row * a.d + col] * phi : 0.0;
    }
#pragma unroll
    for (int rr = 0; rr < kRomRows; ++rr)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part[rr] += __shfl_down_sync(0xffffffffu, part[rr], o);
    if (tid % 32 == 0)
#pragma unroll
        for (int rr = 0; rr < kRomRows; ++rr) red[tid / 32][rr] = part[rr];
    __syncthreads();
    if (tid < kRomRows) {
        const int row = blockIdx.y * kRomRows + tid;
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < kRomBlock / 32; ++w) s += red[w][tid];
        if (row < a.r) a.partial[(long long)blockIdx.x * a.r + row] = s;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const unsigned int ticket = atomicAdd(a.counter, 1u);
        last_block = ticket == gridDim.x * gridDim.y - 1;
    }
    __syncthreads();
    if (!last_block) return;
    __threadfence();
    for (int row = tid; row < a.r; row += blockDim.x) {
        double acc = 0.0;
        for (int bx = 0; bx < (int)gridDim.x; ++bx) acc += __ldcg(a.partial + (long long)bx * a.r + row);
        if (a.rhs_only) {
            a.q[2 * a.r + row] = acc;
        } else {
            const double qd = fma(0.5 * dt, a.q[2 * a.r + row] + acc, a.q[a.r + row]);
            a.q[row] = qp[row];
            a.q[a.r + row] = qd;
            a.q[2 * a.r + row] = acc;
            if (a.qrec) {
                a.qrec[row] = qp[row];
                a.qrec[a.r + row] = qd;
                a.qrec[2 * a.r + row] = acc;
            }
        }
    }
    if (tid == 0) *a.counter = 0u;
}

// out[slot][f][3 i + c] = sum_k Rt[k][3 i + c] q_src[slot][f][k] written into the destination
// history; one thread per (3 i + c), blocks over (column tile, slot, field)
__global__ void k_rom_reconstruct(int nrow, int r, const double* Rt, const double* qsrc, long long qslot_stride,
                                  const int* row, bool dst_rom, double* hist, int nd, int slot0) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    const int slot = slot0 + blockIdx.y;
    const int f = blockIdx.z;
    if (col >= 3 * nrow) return;
    const double* q = qsrc + (long long)blockIdx.y * qslot_stride + (long long)f * r;
    double acc = 0.0;
    for (int k = 0; k < r; ++k) acc = fma(Rt[(long long)k * 3 * nrow + col], q[k], acc);
    const int i = col / 3, c = col % 3;
    const long long idx = dst_rom ? ((long long)(slot * 3 + f) * nd + 3 * row[i] + c)
                                  : ((long long)((slot * 3 + f) * 3 + c) * nd + row[i]);
    hist[idx] = acc;
}

__global__ void k_rom_norms(int r, double dt, const double* q, double* pq, double* partial) {
    double num = 0.0, den = 0.0;
    for (int k = threadIdx.x; k < r; k += blockDim.x) {
        const double x = (q[k] - pq[k]) + dt * (q[r + k] - pq[r + k]);
        const double y = fma(dt, q[r + k], q[k]);
        num = fma(x, x, num);
        den = fma(y, y, den);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < r; k += blockDim.x) {
        pq[k] = q[k];
        pq[r + k] = q[r + k];
    }
    num = block_sum(num);
    __syncthreads();
    den = block_sum(den);
    if (threadIdx.x == 0) {
        partial[0] = num;
        partial[1] = den;
    }
}

// q[f][k] = sum_free Phi[m][k] x_f[free_dof[m]] for f = 0 (u) and 1 (v); one block per (k, f)
__global__ void k_basis_project(int nfree, int r, const double* Phi, const int* free_dof, const double* u_aos,
                                const double* v_aos, double* q) {
    const int k = blockIdx.x;
    const double* x = blockIdx.y == 0 ? u_aos : v_aos;
    double acc = 0.0;
    if (x)
        for (int m = threadIdx.x; m < nfree; m += blockDim.x) acc = fma(Phi[(long long)m * r + k], x[free_dof[m]], acc);
    acc = block_sum(acc);
    if (threadIdx.x == 0 && x) q[blockIdx.y * r + k] = acc;
}

// reconstructed full field [nodes][3]: Phi qv on free dofs, history data on Schwarz nodes, 0 clamped
__global__ void k_full_field(int nn, int r, const double* Phi, const int* dof_free, const uint8_t* clamp,
                             const int* srow, const double* hist_slot_field, int nsdof, const double* qv, double* out) {
    const int dof = blockIdx.x * blockDim.x + threadIdx.x;
    if (dof >= 3 * nn) return;
    const int n = dof / 3, c = dof % 3;
    double val = 0.0;
    if (clamp[n] & (1 << c)) val = 0.0;
    else if (srow[n] >= 0) val = hist_slot_field ? hist_slot_field[3 * srow[n] + c] : 0.0;
    else {
        const int m = dof_free[dof];
        for (int k = 0; k < r; ++k) val = fma(Phi[(long long)m * r + k], qv[k], val);
    }
    out[dof] = val;
}

// Rt[k][3 i + c] = sum_b w_b Phi[free(dnode_b, c)][k]; a donor with nonzero weight on a constrained
// Schwarz dof of the ROM is rejected (err)
__global__ void k_build_Rt(int nrow, int r, const int* dnode, const double* dw, const int* dof_free,
                           const int* srow, const double* Phi, double* Rt, int* err) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (col >= 3 * nrow) return;
    const int i = col / 3, c = col % 3;
    double acc = 0.0;
    for (int b = 0; b < 8; ++b) {
        const double w = dw[8 * i + b];
        if (w == 0.0) continue;
        const int n = dnode[8 * i + b];
        const int m = dof_free[3 * n + c];
        if (m >= 0) acc = fma(w, Phi[(long long)m * r + k], acc);
        else if (srow[n] >= 0 && k == 0) atomicAdd(err, 1);
    }
    Rt[(long long)k * 3 * nrow + col] = acc;
}

// generic FP64 GEMM C(i,j) = alpha sum_k A(i,k) B(k,j) + beta C(i,j) with element strides
constexpr int TM = 64, TN = 64, TK = 16;
__global__ void __launch_bounds__(256) k_gemm(int m, int n, int kdim, const double* A, long long ai, long long ak,
                                              const double* B, long long bk, long long bj, double* C, long long ldc,
                                              double alpha, double beta) {
    __shared__ double As[TK][TM + 1];
    __shared__ double Bs[TK][TN + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int i0 = blockIdx.y * TM, j0 = blockIdx.x * TN;
    double acc[4][4] = {{0}};
    for (int k0 = 0; k0 < kdim; k0 += TK) {
        for (int t = threadIdx.x; t < TK * TM; t += 256) {
            const int kk = t % TK, ii = t / TK;
            const int gi = i0 + ii, gk = k0 + kk;
            As[kk][ii] = (gi < m && gk < kdim) ? A[gi * ai + gk * ak] : 0.0;
        }
        for (int t = threadIdx.x; t < TK * TN; t += 256) {
            const int jj = t % TN, kk = t / TN;
            const int gj = j0 + jj, gk = k0 + kk;
            Bs[kk][jj] = (gj < n && gk < kdim) ? B[gk * bk + gj * bj] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            double a4[4], b4[4];
#pragma unroll
            for (int x = 0; x < 4; ++x) { a4[x] = As[kk][ty * 4 + x]; b4[x] = Bs[kk][tx * 4 + x]; }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fma(a4[x], b4[y], acc[x][y]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const int gi = i0 + ty * 4 + x, gj = j0 + tx * 4 + y;
            if (gi < m && gj < n) {
                double* cp = C + gi * ldc + gj;
                *cp = alpha * acc[x][y] + (beta != 0.0 ? beta * *cp : 0.0);
            }
        }
}

// compressed Kronecker features: D[s][col0 + idx(i,j)] = Ubar[i][s] * Ubar[j][s] (i <= j)
__global__ void k_kron_features(const double* Ubar, int r, int nsnap, double* D, int ldd, int col0) {
    const int s = blockIdx.x;
    int idx = 0;
    for (int i = 0; i < r; ++i) {
        const double qi = Ubar[(long long)i * nsnap + s];
        for (int j = i + threadIdx.x; j < r; j += blockDim.x)
            D[(long long)s * ldd + col0 + idx + (j - i)] = qi * Ubar[(long long)j * nsnap + s];
        idx += r - i;
    }
}

}  // namespace

cudaError_t launch_rom_project(const RomDev& r, int slot0, int slot1, cudaStream_t s) {
    if (r.rs == 0 || slot1 < slot0) return cudaSuccess;
    dim3 g(r.rs, slot1 - slot0 + 1);
    k_rom_project<<<g, 128, 0, s>>>(r.PhiSt, r.hist, r.ghat, r.rs, r.nsdof, slot0);
    return cudaGetLastError();
}

cudaError_t launch_rom_step(const RomDev& r, int slot, double dt, int rhs_only, cudaStream_t s) {
    if (r.r > kMaxR) return cudaErrorInvalidValue;
    RomStepArgs a;
    a.r = r.r; a.d = r.d; a.nq = r.nq; a.rs = r.rs;
    a.O = r.O; a.kij = r.kron_ij; a.q = r.q;
    a.ghat = r.ghat + (long long)slot * r.rs;
    a.dt = dt;
    a.partial = r.partial;
    a.counter = r.counter;
    a.qrec = rhs_only ? nullptr : r.qrec + (long long)slot * 3 * r.r;
    a.rhs_only = rhs_only;
    dim3 g(grid_for(r.d, kRomBlock), grid_for(r.r, kRomRows));
    k_rom_step<<<g, kRomBlock, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_rom_reconstruct(const CplDev& c, const RomDev& src, bool zoh, bool dst_rom, double* dst_hist,
                                   int nd, int nsub, cudaStream_t s) {
    if (c.nrow == 0) return cudaSuccess;
    if (zoh) {
        // the current reduced state, written to every slot
        dim3 g(grid_for(3LL * c.nrow, 128), nsub + 1, 3);
        k_rom_reconstruct<<<g, 128, 0, s>>>(c.nrow, src.r, c.Rt, src.q, 0, c.row, dst_rom, dst_hist, nd, 0);
    } else {
        dim3 g(grid_for(3LL * c.nrow, 128), nsub, 3);
        k_rom_reconstruct<<<g, 128, 0, s>>>(c.nrow, src.r, c.Rt, src.qrec + 3LL * src.r, 3LL * src.r, c.row, dst_rom,
                                            dst_hist, nd, 1);
    }
    return cudaGetLastError();
}

cudaError_t launch_rom_norms(const RomDev& r, double dt, double* partial, cudaStream_t s) {
    k_rom_norms<<<1, 128, 0, s>>>(r.r, dt, r.q, r.pq, partial);
    return cudaGetLastError();
}

cudaError_t launch_rom_basis_project(const RomDev& r, const double* u_aos, const double* v_aos, cudaStream_t s) {
    dim3 g(r.r, 2);
    k_basis_project<<<g, 256, 0, s>>>(r.nfree, r.r, r.Phi, r.free_dof, u_aos, v_aos, r.q);
    return cudaGetLastError();
}

cudaError_t launch_rom_full_field(const RomDev& r, const double* qv, int field, double* out_aos, int slot,
                                  cudaStream_t s) {
    const int nn = r.g.nn();
    const double* hs = r.hist ? r.hist + ((long long)slot * 3 + field) * r.nsdof : nullptr;
    k_full_field<<<grid_for(3LL * nn, 256), 256, 0, s>>>(nn, r.r, r.Phi, r.dof_free, r.clamp, r.srow, hs, r.nsdof, qv,
                                                         out_aos);
    return cudaGetLastError();
}

cudaError_t launch_build_Rt_checked(const CplDev& c, const RomDev& src, int* err, cudaStream_t s) {
    if (c.nrow == 0) return cudaSuccess;
    dim3 g(grid_for(3LL * c.nrow, 128), src.r);
    k_build_Rt<<<g, 128, 0, s>>>(c.nrow, src.r, c.dnode, c.dw, src.dof_free, src.srow, src.Phi, c.Rt, err);
    return cudaGetLastError();
}

// row-major helpers: C[m][n] (ldc) = alpha * A^T B, A is [k][m] (lda), B is [k][n] (ldb)
cudaError_t launch_gemm_tn(int m, int n, int k, const double* A, int lda, const double* B, int ldb, double* C, int ldc,
                           double alpha, double beta, cudaStream_t s) {
    dim3 g(grid_for(n, TN), grid_for(m, TM));
    k_gemm<<<g, 256, 0, s>>>(m, n, k, A, 1, lda, B, ldb, 1, C, ldc, alpha, beta);
    return cudaGetLastError();
}

// C[m][n] = alpha * A B, A is [m][k] (lda), B is [k][n] (ldb)
cudaError_t launch_gemm_nn(int m, int n, int k, const double* A, int lda, const double* B, int ldb, double* C, int ldc,
                           double alpha, double beta, cudaStream_t s) {
    dim3 g(grid_for(n, TN), grid_for(m, TM));
    k_gemm<<<g, 256, 0, s>>>(m, n, k, A, lda, 1, B, ldb, 1, C, ldc, alpha, beta);
    return cudaGetLastError();
}

// C[m][n] = alpha * A B^T, A is [m][k] (lda), B is [n][k] (ldb)
cudaError_t launch_gemm_nt(int m, int n, int k, const double* A, int lda, const double* B, int ldb, double* C, int ldc,
                           double alpha, double beta, cudaStream_t s) {
    dim3 g(grid_for(n, TN), grid_for(m, TM));
    k_gemm<<<g, 256, 0, s>>>(m, n, k, A, lda, 1, B, 1, ldb, C, ldc, alpha, beta);
    return cudaGetLastError();
}

cudaError_t launch_kron_features(const double* Ubar, int r, int nsnap, double* D, int ldd, int col0, cudaStream_t s) {
    k_kron_features<<<nsnap, 64, 0, s>>>(Ubar, r, nsnap, D, ldd, col0);
    return cudaGetLastError();
}

}  // namespace osam
