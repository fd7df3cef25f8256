// FOM set-up and I/O kernels, and the element-level internal-force kernel of the C ABI
// (osam_hex8_force / osam_hex8_force_noalloc).  The per-step kernels of the controller, which work
// on every instance of a batch at once, are in step_kernels.cu; both use hex8_math.cuh.
#include <cuda_runtime.h>

#include <cstdint>

#include "hex8_math.cuh"
#include "osam_internal.h"

namespace osam {

namespace {

using namespace hex8;

// one thread per element of a single mesh, strided input / output (see ElemArgs)
template <int MAT, typename T, int MODE>
__global__ void __launch_bounds__(128) k_hex8_force(const ElemArgs a) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.ne) return;
    const int i = e % a.nx;
    const int t = e / a.nx;
    const int j = t % a.ny;
    const int k = t / a.ny;
    const int sy = a.nx + 1, sz = (a.nx + 1) * (a.ny + 1);
    const int n0 = i + sy * j + sz * k;
    int node[8];
#pragma unroll
    for (int c8 = 0; c8 < 8; ++c8) node[c8] = n0 + (c8 & 1) + ((c8 >> 1) & 1) * sy + ((c8 >> 2) & 1) * sz;
    const double lam = a.lam_e ? a.lam_e[e] : a.lam;
    const double mu = a.mu_e ? a.mu_e[e] : a.mu;
    T m1, m2, m3;
    material_factors<MAT, T>(lam, mu, a.wq, a.wq3, m1, m2, m3);
    T Dx[3][2][2], Dy[3][2][2], Dz[3][2][2];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double U[8];
        const double* uc = a.u + (long long)c * a.usc;
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8) U[c8] = uc[(long long)node[c8] * a.usn];
        edge_differences<T>(U, a.invh, Dx[c], Dy[c], Dz[c]);
    }
    T F[3][8];
    element_force<MAT, T>(Dx, Dy, Dz, m1, m2, m3, F);
    if (MODE == kAtomic) {
        T* f = static_cast<T*>(a.f);
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int c8 = 0; c8 < 8; ++c8) atomic_add(f + (long long)c * a.fsc + (long long)node[c8] * a.fsn, F[c][c8]);
    } else {
        T* fe = static_cast<T*>(a.fe);
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8)
#pragma unroll
            for (int c = 0; c < 3; ++c) fe[(long long)(c8 * 3 + c) * a.ne + e] = F[c][c8];
    }
}

// inverse row-sum lumped mass of a uniform cubic mesh: m_n = rho h^3 / 8 x (adjacent elements)
__global__ void k_lumped_minv(int nx, int ny, int nz, double m_e8, double* minv, double* mass) {
    const int nn = (nx + 1) * (ny + 1) * (nz + 1);
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nn) return;
    const int i = n % (nx + 1);
    const int t = n / (nx + 1);
    const int j = t % (ny + 1);
    const int k = t / (ny + 1);
    const int cx = (i > 0) + (i < nx), cy = (j > 0) + (j < ny), cz = (k > 0) + (k < nz);
    const double m = m_e8 * double(cx * cy * cz);
    minv[n] = 1.0 / m;
    if (mass) mass[n] = m;
}

// donor element and trilinear weights of each destination Schwarz node in a structured source box:
// lowest-index element containing the point, local coordinates within 1e-9 of +-1 snapped to +-1.
// dnode receives node indices local to the source mesh.
__global__ void k_donor(Grid src, Grid dst, const int* dst_nodes, int nrow, int* dnode, double* dw, int* err) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nrow) return;
    const int n = dst_nodes[t];
    int idx[3] = {n % (dst.nx + 1), (n / (dst.nx + 1)) % (dst.ny + 1), n / ((dst.nx + 1) * (dst.ny + 1))};
    const int ns[3] = {src.nx, src.ny, src.nz};
    int el[3];
    double xi[3];
    for (int ax = 0; ax < 3; ++ax) {
        const double x = dst.org[ax] + idx[ax] * dst.h;
        const double tt = (x - src.org[ax]) / src.h;
        int found = -1;
        double xf = 0.0;
        const int base = (int)floor(tt);
        for (int cand = base - 1; cand <= base + 1; ++cand) {
            if (cand < 0 || cand >= ns[ax]) continue;
            const double xc = 2.0 * (tt - cand) - 1.0;
            if (fabs(xc) <= 1.0 + 1e-9) { found = cand; xf = xc; break; }
        }
        if (found < 0) { atomicAdd(err, 1); el[ax] = 0; xi[ax] = 0.0; continue; }
        if (fabs(xf - 1.0) <= 1e-9) xf = 1.0;
        if (fabs(xf + 1.0) <= 1e-9) xf = -1.0;
        el[ax] = found;
        xi[ax] = xf;
    }
    const int sy = src.nx + 1, sz = (src.nx + 1) * (src.ny + 1);
    const int n0 = el[0] + sy * el[1] + sz * el[2];
    for (int c8 = 0; c8 < 8; ++c8) {
        const int bx = c8 & 1, by = (c8 >> 1) & 1, bz = (c8 >> 2) & 1;
        dnode[8 * t + c8] = n0 + bx + by * sy + bz * sz;
        const double sxv = bx ? 1.0 : -1.0, syv = by ? 1.0 : -1.0, szv = bz ? 1.0 : -1.0;
        dw[8 * t + c8] = 0.125 * (1.0 + sxv * xi[0]) * (1.0 + syv * xi[1]) * (1.0 + szv * xi[2]);
    }
}

// interleaved [nn][3] <-> component-strided soa[c * stride + n]
__global__ void k_aos_to_soa(const double* aos, double* soa, int nn, long long stride) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * nn) return;
    const int n = t / 3, c = t % 3;
    soa[(long long)c * stride + n] = aos[t];
}

__global__ void k_soa_to_aos(const double* soa, double* aos, int nn, long long stride) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * nn) return;
    const int n = t / 3, c = t % 3;
    aos[t] = soa[(long long)c * stride + n];
}

__global__ void k_zero_clamped(int nn, const uint8_t* clamp, double* u, double* v, long long stride) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * nn) return;
    const int c = t / nn, n = t % nn;
    if (clamp[n] & (1 << c)) {
        u[(long long)c * stride + n] = 0.0;
        if (v) v[(long long)c * stride + n] = 0.0;
    }
}


// Stiffest element modulus of each instance for the explicit stability check.  A cube element with
// 2x2x2 Gauss points has the largest stiffness eigenvalue h max(3/2 lambda + mu, mu); with the lumped
// element mass rho h^3 / 8 per node that bounds omega_max^2 by 8 max(3/2 lambda + mu, mu) / (rho h^2)
// (the element eigenvalue inequality), so the stable step is h sqrt(rho / max(3 lambda + 2 mu, 2 mu)).
// out[inst] receives the bits of the largest max(3 lambda_e + 2 mu_e, 2 mu_e) (non-negative doubles
// order like their bit patterns); *bad is set for a material that is not positive definite.
__global__ void k_cfl_modulus(const FomB g, unsigned long long* out, int* bad) {
    const int2 b = g.eblk[blockIdx.x];
    const InstFom I = g.inst[b.x];
    const int e = b.y + (int)threadIdx.x;
    double m = 0.0;
    if ((int)threadIdx.x < g.eblock && e < I.ne) {
        const double lam = I.lam_e ? I.lam_e[e] : I.lam;
        const double mu = I.mu_e ? I.mu_e[e] : I.mu;
        const double p = 3.0 * lam + 2.0 * mu;
        if (!(mu > 0.0) || !(p > 0.0) || !isfinite(p)) *bad = 1;
        else m = fmax(p, 2.0 * mu);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(out + b.x, (unsigned long long)__double_as_longlong(m));
}

}  // namespace

int grid_for(long long n, int block) { return (int)((n + block - 1) / block); }

cudaError_t launch_hex8_force(int material, bool fp32, int scatter, const ElemArgs& a, cudaStream_t s) {
    if (a.ne <= 0) return cudaSuccess;
    const int g = grid_for(a.ne, 128);
#define OSAM_LAUNCH(MAT, T, MODE) k_hex8_force<MAT, T, MODE><<<g, 128, 0, s>>>(a)
    if (material == OSAM_NEO_HOOKEAN) {
        if (fp32) { if (scatter == kAtomic) OSAM_LAUNCH(OSAM_NEO_HOOKEAN, float, kAtomic); else OSAM_LAUNCH(OSAM_NEO_HOOKEAN, float, kGather); }
        else { if (scatter == kAtomic) OSAM_LAUNCH(OSAM_NEO_HOOKEAN, double, kAtomic); else OSAM_LAUNCH(OSAM_NEO_HOOKEAN, double, kGather); }
    } else if (material == OSAM_SAINT_VENANT_KIRCHHOFF) {
        if (fp32) { if (scatter == kAtomic) OSAM_LAUNCH(OSAM_SAINT_VENANT_KIRCHHOFF, float, kAtomic); else OSAM_LAUNCH(OSAM_SAINT_VENANT_KIRCHHOFF, float, kGather); }
        else { if (scatter == kAtomic) OSAM_LAUNCH(OSAM_SAINT_VENANT_KIRCHHOFF, double, kAtomic); else OSAM_LAUNCH(OSAM_SAINT_VENANT_KIRCHHOFF, double, kGather); }
    } else {
        if (fp32) { if (scatter == kAtomic) OSAM_LAUNCH(OSAM_LINEAR_ELASTIC, float, kAtomic); else OSAM_LAUNCH(OSAM_LINEAR_ELASTIC, float, kGather); }
        else { if (scatter == kAtomic) OSAM_LAUNCH(OSAM_LINEAR_ELASTIC, double, kAtomic); else OSAM_LAUNCH(OSAM_LINEAR_ELASTIC, double, kGather); }
    }
#undef OSAM_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_lumped_minv(const Grid& g, double rho, double* minv, cudaStream_t s, double* mass) {
    const double m_e8 = rho * g.h * g.h * g.h / 8.0;
    k_lumped_minv<<<grid_for(g.nn(), 256), 256, 0, s>>>(g.nx, g.ny, g.nz, m_e8, minv, mass);
    return cudaGetLastError();
}

cudaError_t launch_donor(const Grid& src, const Grid& dst, const int* dst_nodes, int nrow, int* dnode, double* dw,
                         int* err, cudaStream_t s) {
    if (nrow == 0) return cudaSuccess;
    k_donor<<<grid_for(nrow, 128), 128, 0, s>>>(src, dst, dst_nodes, nrow, dnode, dw, err);
    return cudaGetLastError();
}

cudaError_t launch_aos_to_soa(const double* aos, double* soa, int nn, long long stride, cudaStream_t s) {
    k_aos_to_soa<<<grid_for(3LL * nn, 256), 256, 0, s>>>(aos, soa, nn, stride);
    return cudaGetLastError();
}

cudaError_t launch_soa_to_aos(const double* soa, double* aos, int nn, long long stride, cudaStream_t s) {
    k_soa_to_aos<<<grid_for(3LL * nn, 256), 256, 0, s>>>(soa, aos, nn, stride);
    return cudaGetLastError();
}

cudaError_t launch_cfl_modulus(const FomB& g, unsigned long long* out, int* bad, cudaStream_t s) {
    if (g.n_eblk == 0) return cudaSuccess;
    const int threads = (g.eblock + 31) / 32 * 32;
    k_cfl_modulus<<<g.n_eblk, threads, 0, s>>>(g, out, bad);
    return cudaGetLastError();
}

cudaError_t launch_zero_clamped(int nn, const uint8_t* clamp, double* u, double* v, long long stride, cudaStream_t s) {
    k_zero_clamped<<<grid_for(3LL * nn, 256), 256, 0, s>>>(nn, clamp, u, v, stride);
    return cudaGetLastError();
}

}  // namespace osam
