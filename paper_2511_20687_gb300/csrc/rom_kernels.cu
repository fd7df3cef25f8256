// OpInf ROM set-up and I/O kernels (Sec. 4.2): basis projection q = Phi^T u, full-field
// reconstruction, the reconstruction operator (Pi Phi_rows)^T of a ROM source, and the dense FP64
// products of the offline fit.  The per-step ROM kernels are in step_kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "osam_internal.h"

namespace osam {

namespace {

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

// generic FP64 GEMM C(i,j) = alpha sum_k A(i,k) B(k,j) + beta C(i,j) with element strides.
// The tile loaders walk the operand along its contiguous index (k for a row-major A, i for a
// transposed one; likewise j or k for B), so every warp reads whole 128-byte lines.  With split-K
// (gridDim.z > 1) block z sums k in [z kchunk, (z + 1) kchunk) and stores its partial tile into
// ws[z][m][n]; k_gemm_reduce then adds the partials in ascending z (deterministic) and applies
// alpha and beta.  The output tiles are numbered along grid.x, column tile fastest (blocks that
// share a row tile of A run together and find it in L2), so m is bounded only by 32-bit indices.
constexpr int TM = 64, TN = 64, TK = 16;

// The GEMM runs on the FP64 tensor cores: 128 threads per 64x64 output tile, each warp a 32x32 quarter
// as 4 x 4 accumulators of mma.sync m8n8k4 (FP64 in and out, each MMA 8x8x4 fused multiply-adds).
// Fragments (groupID g = lane / 4, t = lane % 4): A element (row g, k t), B element (k t, col g),
// accumulator elements (row g, cols 2t, 2t + 1).  Shared-memory rows padded to 68 doubles so that the
// 16 lanes of each half-warp read distinct banks.
constexpr int TPAD = 4;
__device__ __forceinline__ void dmma_8x8x4(double& d0, double& d1, double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
                 : "+d"(d0), "+d"(d1)
                 : "d"(a), "d"(b));
}

__global__ void __launch_bounds__(128) k_gemm_mma(int m, int n, int kdim, int kchunk, const double* A, long long ai,
                                                  long long ak, const double* B, long long bk, long long bj,
                                                  double* C, long long ldc, double alpha, double beta, double* ws) {
    __shared__ double As[TK][TM + TPAD];
    __shared__ double Bs[TK][TN + TPAD];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wr = warp >> 1, wc = warp & 1;
    const int g = lane >> 2, t4 = lane & 3;
    const int ntn = (n + TN - 1) / TN;
    const int i0 = (int)(blockIdx.x / ntn) * TM, j0 = (int)(blockIdx.x % ntn) * TN;
    const int kbeg = blockIdx.z * kchunk;
    const int kend = min(kdim, kbeg + kchunk);
    const bool a_along_i = ai == 1 && ak != 1;   // A stored [k][m]
    const bool b_along_j = bj == 1;              // B stored [k][n]
    double acc[4][4][2];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y][0] = acc[x][y][1] = 0.0;
    for (int k0 = kbeg; k0 < kend; k0 += TK) {
        for (int t = threadIdx.x; t < TK * TM; t += 128) {
            const int kk = a_along_i ? t / TM : t % TK, ii = a_along_i ? t % TM : t / TK;
            const int gi = i0 + ii, gk = k0 + kk;
            As[kk][ii] = (gi < m && gk < kend) ? A[gi * ai + gk * ak] : 0.0;
        }
        for (int t = threadIdx.x; t < TK * TN; t += 128) {
            const int jj = b_along_j ? t % TN : t / TK, kk = b_along_j ? t / TN : t % TK;
            const int gj = j0 + jj, gk = k0 + kk;
            Bs[kk][jj] = (gj < n && gk < kend) ? B[gk * bk + gj * bj] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < TK; ks += 4) {
            double a[4], b[4];
#pragma unroll
            for (int x = 0; x < 4; ++x) a[x] = As[ks + t4][wr * 32 + x * 8 + g];
#pragma unroll
            for (int y = 0; y < 4; ++y) b[y] = Bs[ks + t4][wc * 32 + y * 8 + g];
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) dmma_8x8x4(acc[x][y][0], acc[x][y][1], a[x], b[y]);
        }
        __syncthreads();
    }
    double* W = ws ? ws + (long long)blockIdx.z * m * n : nullptr;
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int gi = i0 + wr * 32 + x * 8 + g, gj = j0 + wc * 32 + y * 8 + 2 * t4 + q;
                if (gi < m && gj < n) {
                    if (W) {
                        W[(long long)gi * n + gj] = acc[x][y][q];
                    } else {
                        double* cp = C + gi * ldc + gj;
                        *cp = alpha * acc[x][y][q] + (beta != 0.0 ? beta * *cp : 0.0);
                    }
                }
            }
}

__global__ void k_gemm_reduce(int m, int n, int nsplit, const double* __restrict__ ws, double* C, long long ldc,
                              double alpha, double beta) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long mn = (long long)m * n;
    if (idx >= mn) return;
    double s = 0.0;
    for (int z = 0; z < nsplit; ++z) s += ws[z * mn + idx];
    double* cp = C + (idx / n) * ldc + idx % n;
    *cp = alpha * s + (beta != 0.0 ? beta * *cp : 0.0);
}

// Optional accounting of the fit's contractions (osam_fit_profile): CUDA events around every GEMM
// (both kernels of a split reduction), its 2 m n k flops, per host thread.  Off by default; when on,
// each GEMM waits for its end event, so the fit runs slower than without it.
struct GemmProfile {
    bool on = false;
    double ms = 0.0, flops = 0.0;
    long long launches = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
};
thread_local GemmProfile g_gemm_prof;

cudaError_t launch_gemm_impl(int m, int n, int k, const double* A, long long ai, long long ak, const double* B,
                             long long bk, long long bj, double* C, long long ldc, double alpha, double beta,
                             cudaStream_t s);

cudaError_t launch_gemm(int m, int n, int k, const double* A, long long ai, long long ak, const double* B,
                        long long bk, long long bj, double* C, long long ldc, double alpha, double beta,
                        cudaStream_t s) {
    GemmProfile& P = g_gemm_prof;
    if (!P.on || m <= 0 || n <= 0) return launch_gemm_impl(m, n, k, A, ai, ak, B, bk, bj, C, ldc, alpha, beta, s);
    cudaError_t e = cudaEventRecord(P.e0, s);
    if (e == cudaSuccess) e = launch_gemm_impl(m, n, k, A, ai, ak, B, bk, bj, C, ldc, alpha, beta, s);
    if (e == cudaSuccess) e = cudaEventRecord(P.e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(P.e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, P.e0, P.e1);
    if (e == cudaSuccess) {
        P.ms += ms;
        P.flops += 2.0 * m * (double)n * k;
        P.launches += 1;
    }
    return e;
}

// Split the reduction when the output tiles alone cannot fill the GPU (four 4-warp blocks per SM
// wanted) and the reduction is long: chunks of at least 512 k, a multiple of the k tile.
cudaError_t launch_gemm_impl(int m, int n, int k, const double* A, long long ai, long long ak, const double* B,
                             long long bk, long long bj, double* C, long long ldc, double alpha, double beta,
                             cudaStream_t s) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    const long long tiles = (long long)grid_for(n, TN) * grid_for(m, TM);
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = 4LL * sms;
    int nsplit = 1;
    if (tiles < want && k >= 2 * 512)
        nsplit = (int)std::min<long long>((want + tiles - 1) / tiles, k / 512);
    // prefer a block count that is a multiple of the SM count: every SM then runs the same number of
    // equal blocks (a 64-tile Gram split 10 ways leaves some SMs three blocks and others two)
    if (nsplit > 1)
        for (long long ns = nsplit; ns <= std::min<long long>(k / 512, 4LL * nsplit); ++ns)
            if ((tiles * ns) % sms == 0) { nsplit = (int)ns; break; }
    int kchunk = k;
    if (nsplit > 1) {
        kchunk = (k + nsplit - 1) / nsplit;
        kchunk = (kchunk + TK - 1) / TK * TK;
        nsplit = (k + kchunk - 1) / kchunk;
    }
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    dim3 g((unsigned)tiles, 1, nsplit);
    if (nsplit == 1) {
        k_gemm_mma<<<g, 128, 0, s>>>(m, n, k, k, A, ai, ak, B, bk, bj, C, ldc, alpha, beta, nullptr);
        return cudaGetLastError();
    }
    double* ws = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&ws), sizeof(double) * (size_t)nsplit * m * n, s);
    if (e != cudaSuccess) return e;
    k_gemm_mma<<<g, 128, 0, s>>>(m, n, k, kchunk, A, ai, ak, B, bk, bj, C, ldc, alpha, beta, ws);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        k_gemm_reduce<<<grid_for((long long)m * n, 256), 256, 0, s>>>(m, n, nsplit, ws, C, ldc, alpha, beta);
        e = cudaGetLastError();
    }
    cudaError_t f = cudaFreeAsync(ws, s);
    return e != cudaSuccess ? e : f;
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


// compressed Kronecker cube: one block per snapshot, index triples (i <= j <= k) in lexicographic order
__global__ void k_kron3_features(const double* Ubar, int r, int nsnap, double* D, int ldd, int col0) {
    const int s = blockIdx.x;
    long long idx = 0;
    for (int i = 0; i < r; ++i) {
        const double qi = Ubar[(long long)i * nsnap + s];
        for (int j = i; j < r; ++j) {
            const double qij = qi * Ubar[(long long)j * nsnap + s];
            for (int k = j + threadIdx.x; k < r; k += blockDim.x)
                D[(long long)s * ldd + col0 + idx + (k - j)] = qij * Ubar[(long long)k * nsnap + s];
            idx += r - j;
        }
    }
}

// Regularisation selection (Sec. 4.2.4, Algorithm 3): one block per candidate lambda rolls its ROM
// out alone, explicit central differences with step dt, Schwarz boundary data frozen to the training
// columns (linear in time between columns that are k steps apart), from the training initial state;
// accumulates ||q(t_j) - Ubar_j||^2 and ||Ubar_j||^2 over the snapshot times in a fixed order.
constexpr int kSelBlock = 256;
constexpr int kSelMaxR = 128;

__device__ __forceinline__ double2 block_sum_pair(double x, double y) {
    __shared__ double sx[kSelBlock / 32], sy[kSelBlock / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_down_sync(0xffffffffu, x, o);
        y += __shfl_down_sync(0xffffffffu, y, o);
    }
    const int w = threadIdx.x / 32, ln = threadIdx.x % 32;
    __syncthreads();
    if (ln == 0) { sx[w] = x; sy[w] = y; }
    __syncthreads();
    double a = 0.0, b = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x / 32); ++i) { a += sx[i]; b += sy[i]; }
    return make_double2(a, b);
}

__global__ void __launch_bounds__(kSelBlock) k_select_rollout(int r, int d, int nq, int nc, int rs,
                                                              const double* __restrict__ O,
                                                              const short2* __restrict__ kij,
                                                              const short4* __restrict__ kijk,
                                                              const double* __restrict__ D,
                                                              const double* __restrict__ Y, const double* __restrict__ qd0,
                                                              int ns, int k, double dt, double* phi_all, double* num,
                                                              double* den) {
    __shared__ double q[kSelMaxR], qd[kSelMaxR], qdd[kSelMaxR], qp[kSelMaxR], qn[kSelMaxR];
    const int l = blockIdx.x, tid = threadIdx.x;
    const double* Ol = O + (size_t)l * r * d;
    double* phi = phi_all + (size_t)l * d;
    const int nwarp = blockDim.x / 32, warp = tid / 32, lane = tid % 32;
    for (int t = tid; t < r; t += blockDim.x) {
        q[t] = D[t];
        qd[t] = qd0[t];
        qdd[t] = Y[t];
    }
    double2 acc = block_sum_pair(0.0, tid < r ? D[tid] * D[tid] : 0.0);
    double sn = 0.0, sd = acc.y;   // meaningful in thread 0
    const double hdt = 0.5 * dt, hdt2 = 0.5 * dt * dt;
    for (int j = 0; j + 1 < ns; ++j) {
        const double* g0 = D + (size_t)j * d + r + nq + nc;
        const double* g1 = D + (size_t)(j + 1) * d + r + nq + nc;
        for (int s = 1; s <= k; ++s) {
            __syncthreads();
            for (int t = tid; t < r; t += blockDim.x) qp[t] = q[t] + dt * qd[t] + hdt2 * qdd[t];
            __syncthreads();
            const double w = (double)s / (double)k;
            for (int col = tid; col < d; col += blockDim.x) {
                double v;
                if (col < r) v = qp[col];
                else if (col < r + nq) { const short2 ij = kij[col - r]; v = qp[ij.x] * qp[ij.y]; }
                else if (col < r + nq + nc) {
                    const short4 t3 = kijk[col - r - nq];
                    v = qp[t3.x] * qp[t3.y] * qp[t3.z];
                }
                else if (col < r + nq + nc + rs) { const int b = col - r - nq - nc; v = g0[b] + w * (g1[b] - g0[b]); }
                else v = 1.0;
                phi[col] = v;
            }
            __syncthreads();
            for (int row = warp; row < r; row += nwarp) {
                const double* orow = Ol + (size_t)row * d;
                double a = 0.0;
                for (int col = lane; col < d; col += 32) a = fma(orow[col], phi[col], a);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
                if (lane == 0) qn[row] = a;
            }
            __syncthreads();
            for (int t = tid; t < r; t += blockDim.x) {
                qd[t] = qd[t] + hdt * (qdd[t] + qn[t]);
                qdd[t] = qn[t];
                q[t] = qp[t];
            }
        }
        __syncthreads();
        double e = 0.0, u = 0.0;
        if (tid < r) {
            const double ub = D[(size_t)(j + 1) * d + tid];
            e = (q[tid] - ub) * (q[tid] - ub);
            u = ub * ub;
        }
        acc = block_sum_pair(e, u);
        sn += acc.x;
        sd += acc.y;
    }
    if (tid == 0) {
        num[l] = sn;
        den[l] = sd;
    }
}

}  // namespace

cudaError_t launch_rom_basis_project(int nfree, int r, const double* Phi, const int* free_dof, const double* u_aos,
                                     const double* v_aos, double* q, cudaStream_t s) {
    dim3 g(r, 2);
    k_basis_project<<<g, 256, 0, s>>>(nfree, r, Phi, free_dof, u_aos, v_aos, q);
    return cudaGetLastError();
}

cudaError_t launch_rom_full_field(int nn, int r, const double* Phi, const int* dof_free, const uint8_t* clamp,
                                  const int* srow, const double* hist_slot_field, const double* qv, double* out_aos,
                                  cudaStream_t s) {
    k_full_field<<<grid_for(3LL * nn, 256), 256, 0, s>>>(nn, r, Phi, dof_free, clamp, srow, hist_slot_field, 0, qv,
                                                         out_aos);
    return cudaGetLastError();
}

cudaError_t launch_build_Rt(int nrow, int r, const int* dnode_local, const double* dw, const int* dof_free,
                            const int* srow, const double* Phi, double* Rt, int* err, cudaStream_t s) {
    if (nrow == 0) return cudaSuccess;
    dim3 g(grid_for(3LL * nrow, 128), r);
    k_build_Rt<<<g, 128, 0, s>>>(nrow, r, dnode_local, dw, dof_free, srow, Phi, Rt, err);
    return cudaGetLastError();
}

int gemm_profile(int enable, double* ms, double* flops, long long* launches) {
    GemmProfile& P = g_gemm_prof;
    if (enable) {
        if (!P.e0 && (cudaEventCreate(&P.e0) != cudaSuccess || cudaEventCreate(&P.e1) != cudaSuccess))
            return OSAM_ECUDA;
        P.ms = 0.0; P.flops = 0.0; P.launches = 0;
    }
    P.on = enable != 0;
    if (ms) *ms = P.ms;
    if (flops) *flops = P.flops;
    if (launches) *launches = P.launches;
    return OSAM_OK;
}

// row-major helpers: C[m][n] (ldc) = alpha * A^T B, A is [k][m] (lda), B is [k][n] (ldb)
cudaError_t launch_gemm_tn(int m, int n, int k, const double* A, int lda, const double* B, int ldb, double* C, int ldc,
                           double alpha, double beta, cudaStream_t s) {
    return launch_gemm(m, n, k, A, 1, lda, B, ldb, 1, C, ldc, alpha, beta, s);
}

// C[m][n] = alpha * A B, A is [m][k] (lda), B is [k][n] (ldb)
cudaError_t launch_gemm_nn(int m, int n, int k, const double* A, int lda, const double* B, int ldb, double* C, int ldc,
                           double alpha, double beta, cudaStream_t s) {
    return launch_gemm(m, n, k, A, lda, 1, B, ldb, 1, C, ldc, alpha, beta, s);
}

// C[m][n] = alpha * A B^T, A is [m][k] (lda), B is [n][k] (ldb)
cudaError_t launch_gemm_nt(int m, int n, int k, const double* A, int lda, const double* B, int ldb, double* C, int ldc,
                           double alpha, double beta, cudaStream_t s) {
    return launch_gemm(m, n, k, A, lda, 1, B, 1, ldb, C, ldc, alpha, beta, s);
}

cudaError_t launch_kron_features(const double* Ubar, int r, int nsnap, double* D, int ldd, int col0, cudaStream_t s) {
    k_kron_features<<<nsnap, 64, 0, s>>>(Ubar, r, nsnap, D, ldd, col0);
    return cudaGetLastError();
}

cudaError_t launch_kron3_features(const double* Ubar, int r, int nsnap, double* D, int ldd, int col0, cudaStream_t s) {
    k_kron3_features<<<nsnap, 64, 0, s>>>(Ubar, r, nsnap, D, ldd, col0);
    return cudaGetLastError();
}

cudaError_t launch_select_rollout(int nl, int r, int d, int nq, int nc, int rs, const double* O, const short2* kij,
                                  const short4* kijk, const double* D, const double* Y, const double* qd0, int ns,
                                  int k, double dt, double* phi, double* num, double* den, cudaStream_t s) {
    if (r > kSelMaxR || r < 1 || nl < 1 || (nc > 0 && !kijk)) return cudaErrorInvalidValue;
    k_select_rollout<<<nl, kSelBlock, 0, s>>>(r, d, nq, nc, rs, O, kij, kijk, D, Y, qd0, ns, k, dt, phi, num, den);
    return cudaGetLastError();
}

}  // namespace osam
