// Double-float ("f32x2") internal force and node update: the element arithmetic in unevaluated sums
// of two floats on the FP32 pipes (df32.cuh), the state and everything else in FP64.  Same
// sum-factorised formulation as the FP64 kernel (hex8_math.cuh).
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "df32.cuh"
#include "osam_internal.h"
#include "trace_item.cuh"

namespace osam {

namespace {

// ------------------------------------------------------------------------------------------------
// FOM internal force in double-float arithmetic (df32.cuh): the same sum-factorised formulation as
// element_force, evaluated on the FP32 pipes (64x the FP64 issue rate of GB300) with ~48-bit
// significands.  Reads the double-float copy of the displacement written by the node kernel and
// writes float2 (hi, lo) element contributions.
// ------------------------------------------------------------------------------------------------
namespace dfk {
using df::f2;
__device__ __forceinline__ f2 G0() { return df::make(0.21132487058639526f, -5.181208351245914e-09f); }
__device__ __forceinline__ f2 G1() { return df::make(0.7886751294136047f, 5.181208351245914e-09f); }
__device__ __forceinline__ f2 GD() { return df::make(0.5773502588272095f, 1.0362416702491828e-08f); }

__device__ __forceinline__ void lerp2(const f2 D[2][2], f2 out[2][2]) {
    f2 E[2][2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const f2 d = df::sub(D[1][e], D[0][e]);
        E[0][e] = df::fma(G0(), d, D[0][e]);
        E[1][e] = df::fma(G1(), d, D[0][e]);
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const f2 d = df::sub(E[q][1], E[q][0]);
        out[q][0] = df::fma(G0(), d, E[q][0]);
        out[q][1] = df::fma(G1(), d, E[q][0]);
    }
}

__device__ __forceinline__ void lerp2T(const f2 S[2][2], f2 out[2][2]) {
    f2 V[2][2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const f2 s = df::add(S[q][0], S[q][1]);
        V[q][0] = df::fma(GD(), S[q][0], df::mul(G0(), s));
        V[q][1] = df::sub(s, V[q][0]);
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const f2 s = df::add(V[0][e], V[1][e]);
        out[0][e] = df::fma(GD(), V[0][e], df::mul(G0(), s));
        out[1][e] = df::sub(s, out[0][e]);
    }
}

__device__ __forceinline__ void stress_le(const f2 H[3][3], f2 lam, f2 mu, f2 P[3][3]) {
    const f2 lt = df::mul(lam, df::add(df::add(H[0][0], H[1][1]), H[2][2]));
    const f2 mu2 = df::add(mu, mu);
#pragma unroll
    for (int c = 0; c < 3; ++c) P[c][c] = df::fma(mu2, H[c][c], lt);
    P[0][1] = P[1][0] = df::mul(mu, df::add(H[0][1], H[1][0]));
    P[0][2] = P[2][0] = df::mul(mu, df::add(H[0][2], H[2][0]));
    P[1][2] = P[2][1] = df::mul(mu, df::add(H[1][2], H[2][1]));
}

// Saint Venant-Kirchhoff stress (see hex8_math.cuh): E = 1/2 (H + H^T + H^T H), P = (I + H) S
__device__ __forceinline__ void stress_svk(const f2 H[3][3], f2 lam, f2 mu, f2 P[3][3]) {
    f2 S[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            f2 c = df::add(H[i][j], H[j][i]);
#pragma unroll
            for (int k = 0; k < 3; ++k) c = df::fma(H[k][i], H[k][j], c);
            S[i][j] = df::make(0.5f * c.h, 0.5f * c.l);  // E (exact halving)
        }
    const f2 lt = df::mul(lam, df::add(df::add(S[0][0], S[1][1]), S[2][2]));
    const f2 mu2 = df::add(mu, mu);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            S[i][j] = i == j ? df::fma(mu2, S[i][j], lt) : df::mul(mu2, S[i][j]);
            if (j != i) S[j][i] = S[i][j];
        }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            f2 p = S[i][j];
#pragma unroll
            for (int k = 0; k < 3; ++k) p = df::fma(H[i][k], S[k][j], p);
            P[i][j] = p;
        }
}

// cofactor form of the Neo-Hookean stress (see hex8_math.cuh)
__device__ __forceinline__ void stress_nh(const f2 H[3][3], f2 kap2, f2 mu, f2 mu3, f2 P[3][3]) {
    f2 F[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) F[i][j] = (i == j) ? df::add(df::one(), H[i][j]) : H[i][j];
    f2 c[3][3];
    c[0][0] = df::sub(df::mul(F[1][1], F[2][2]), df::mul(F[1][2], F[2][1]));
    c[0][1] = df::sub(df::mul(F[1][2], F[2][0]), df::mul(F[1][0], F[2][2]));
    c[0][2] = df::sub(df::mul(F[1][0], F[2][1]), df::mul(F[1][1], F[2][0]));
    c[1][0] = df::sub(df::mul(F[0][2], F[2][1]), df::mul(F[0][1], F[2][2]));
    c[1][1] = df::sub(df::mul(F[0][0], F[2][2]), df::mul(F[0][2], F[2][0]));
    c[1][2] = df::sub(df::mul(F[0][1], F[2][0]), df::mul(F[0][0], F[2][1]));
    c[2][0] = df::sub(df::mul(F[0][1], F[1][2]), df::mul(F[0][2], F[1][1]));
    c[2][1] = df::sub(df::mul(F[0][2], F[1][0]), df::mul(F[0][0], F[1][2]));
    c[2][2] = df::sub(df::mul(F[0][0], F[1][1]), df::mul(F[0][1], F[1][0]));
    const f2 J = df::add(df::add(df::mul(F[0][0], c[0][0]), df::mul(F[0][1], c[0][1])), df::mul(F[0][2], c[0][2]));
    f2 trC = df::mul(F[0][0], F[0][0]);
#pragma unroll
    for (int k = 1; k < 9; ++k) trC = df::fma(F[k / 3][k % 3], F[k / 3][k % 3], trC);
    const f2 J2 = df::mul(J, J);
    const f2 r3 = df::rcbrt(J2);                          // J^-2/3
    const f2 invJ = df::mul(J, df::mul(r3, df::mul(r3, r3)));
    const f2 alpha = df::mul(mu, r3);
    const f2 beta = df::mul(df::sub(df::mul(kap2, df::sub(J2, df::one())), df::mul(df::mul(mu3, r3), trC)), invJ);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) P[i][j] = df::fma(alpha, F[i][j], df::mul(beta, c[i][j]));
}
}  // namespace dfk

// Phased double-float force: (A) edge differences and interpolation to the Gauss points, unrolled,
// the 36 gradient entries parked in shared memory; (B) a rolled loop over the 8 Gauss points with one
// copy of the constitutive code, accumulating the Gauss-point sums of the transposed interpolation in
// shared memory; (C) the transposed interpolation, unrolled.  Keeping the code small keeps it in the
// instruction cache.  Shared memory is private per thread (column tid of a [72][blockDim] array of
// float2), so no barrier is needed.
constexpr int kDfSlots = 72;  // 36 gradient entries + 36 accumulated sums

template <int MAT>
__global__ void __launch_bounds__(128) k_force_df2_b(const FomB g, const int* __restrict__ active,
                                                     const TraceFuse tr) {
    using df::f2;
    extern __shared__ float2 sm[];
    if ((int)blockIdx.x >= g.n_eblk) {
        trace::fused_trace_block(tr, active, g, (int)blockIdx.x - g.n_eblk);
        return;
    }
    const int2 b = g.eblk[blockIdx.x];
    if (active && !active[b.x]) return;
    const InstFom I = g.inst[b.x];
    const int e = b.y + threadIdx.x;
    if (e >= I.ne) return;
    const int nt = blockDim.x, tid = threadIdx.x;
    auto slot = [&](int s) -> float2& { return sm[s * nt + tid]; };
    auto ld = [&](int s) -> f2 { const float2 v = slot(s); return df::make(v.x, v.y); };
    auto st = [&](int s, f2 v) { slot(s) = make_float2(v.h, v.l); };
    const int i = e % I.nx;
    const int t = e / I.nx;
    const int j = t % I.ny;
    const int k = t / I.ny;
    const int sy = I.nx + 1, sz = (I.nx + 1) * (I.ny + 1);
    const int n0 = i + sy * j + sz * k;
    // (A) gradients: slot (dir * 12 + c * 4 + 2 * s0 + s1), dir 0: Gx[c][q][r], 1: Gy[c][p][r], 2: Gz[c][p][q]
    {
        const float2* ub = g.u2 + I.node_off;
#pragma unroll 1
        for (int c = 0; c < 3; ++c) {
            f2 U[8];
#pragma unroll
            for (int c8 = 0; c8 < 8; ++c8) {
                const float2 v = ub[(long long)c * g.NN + n0 + (c8 & 1) + ((c8 >> 1) & 1) * sy + ((c8 >> 2) & 1) * sz];
                U[c8] = df::make(v.x, v.y);
            }
            f2 D[2][2], G[2][2];
#pragma unroll
            for (int dir = 0; dir < 3; ++dir) {
#pragma unroll
                for (int p = 0; p < 2; ++p)
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const int hi = dir == 0 ? 1 + 2 * p + 4 * q : (dir == 1 ? p + 2 + 4 * q : p + 2 * q + 4);
                        const int lo = dir == 0 ? 2 * p + 4 * q : (dir == 1 ? p + 4 * q : p + 2 * q);
                        D[p][q] = df::sub(U[hi], U[lo]);  // the copy holds u / h
                    }
                dfk::lerp2(D, G);
#pragma unroll
                for (int p = 0; p < 2; ++p)
#pragma unroll
                    for (int q = 0; q < 2; ++q) st(dir * 12 + c * 4 + 2 * p + q, G[p][q]);
            }
        }
    }
    // (B) constitutive law at each Gauss point; sums into slots 36 + (dir * 12 + c * 4 + ...)
    {
        const double lam = I.lam_e ? I.lam_e[e] : I.lam;
        const double mu = I.mu_e ? I.mu_e[e] : I.mu;
        f2 m1, m2, m3;
        if (MAT == OSAM_NEO_HOOKEAN) {
            const double kappa = lam + (2.0 / 3.0) * mu;
            m1 = df::from_double(0.5 * kappa * I.w8); m2 = df::from_double(mu * I.w8); m3 = df::from_double(mu * I.w8 / 3.0);
        } else {
            m1 = df::from_double(lam * I.w8); m2 = df::from_double(mu * I.w8); m3 = df::make(0.f, 0.f);
        }
#pragma unroll 1
        for (int gp = 0; gp < 8; ++gp) {
            const int p = gp >> 2, q = (gp >> 1) & 1, r = gp & 1;
            f2 Hm[3][3], P[3][3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                Hm[c][0] = ld(0 * 12 + c * 4 + 2 * q + r);
                Hm[c][1] = ld(1 * 12 + c * 4 + 2 * p + r);
                Hm[c][2] = ld(2 * 12 + c * 4 + 2 * p + q);
            }
            if (MAT == OSAM_NEO_HOOKEAN) dfk::stress_nh(Hm, m1, m2, m3, P);
            else if (MAT == OSAM_SAINT_VENANT_KIRCHHOFF) dfk::stress_svk(Hm, m1, m2, P);
            else dfk::stress_le(Hm, m1, m2, P);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int sx = 36 + 0 * 12 + c * 4 + 2 * q + r;
                const int sy_ = 36 + 1 * 12 + c * 4 + 2 * p + r;
                const int sz_ = 36 + 2 * 12 + c * 4 + 2 * p + q;
                st(sx, p == 0 ? P[c][0] : df::add(ld(sx), P[c][0]));
                st(sy_, q == 0 ? P[c][1] : df::add(ld(sy_), P[c][1]));
                st(sz_, r == 0 ? P[c][2] : df::add(ld(sz_), P[c][2]));
            }
        }
    }
    // (C) transposed interpolation and edge-difference transpose, per component
    float2* fe = static_cast<float2*>(g.fe) + I.elem_off;
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        f2 F[8], S[2][2], Tm[2][2];
#pragma unroll
        for (int s = 0; s < 4; ++s) S[s >> 1][s & 1] = ld(36 + 0 * 12 + c * 4 + s);
        dfk::lerp2T(S, Tm);
#pragma unroll
        for (int ay = 0; ay < 2; ++ay)
#pragma unroll
            for (int az = 0; az < 2; ++az) {
                F[1 + 2 * ay + 4 * az] = Tm[ay][az];
                F[2 * ay + 4 * az] = df::neg(Tm[ay][az]);
            }
#pragma unroll
        for (int s = 0; s < 4; ++s) S[s >> 1][s & 1] = ld(36 + 1 * 12 + c * 4 + s);
        dfk::lerp2T(S, Tm);
#pragma unroll
        for (int ax = 0; ax < 2; ++ax)
#pragma unroll
            for (int az = 0; az < 2; ++az) {
                F[ax + 2 + 4 * az] = df::add(F[ax + 2 + 4 * az], Tm[ax][az]);
                F[ax + 4 * az] = df::sub(F[ax + 4 * az], Tm[ax][az]);
            }
#pragma unroll
        for (int s = 0; s < 4; ++s) S[s >> 1][s & 1] = ld(36 + 2 * 12 + c * 4 + s);
        dfk::lerp2T(S, Tm);
#pragma unroll
        for (int ax = 0; ax < 2; ++ax)
#pragma unroll
            for (int ay = 0; ay < 2; ++ay) {
                F[ax + 2 * ay + 4] = df::add(F[ax + 2 * ay + 4], Tm[ax][ay]);
                F[ax + 2 * ay] = df::sub(F[ax + 2 * ay], Tm[ax][ay]);
            }
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8) fe[(long long)(c8 * 3 + c) * g.NE + e] = make_float2(F[c8].h, F[c8].l);
    }
}

// node kernel of the double-float force: contributions summed in double-float in a fixed order,
// the update in FP64, and the double-float copy of the predicted displacement for the next force
__global__ void __launch_bounds__(kNodeBlock) k_node_df_b(const FomB g, const int* __restrict__ active, int slot1,
                                                         int slot2, int predict_only, const double* ucur,
                                                         double* unext, double dt) {
    using df::f2;
    const int2 b = g.nblk[blockIdx.x];
    if (active && !active[b.x]) return;
    const InstFom I = g.inst[b.x];
    const int n = b.y + threadIdx.x;
    if (n >= I.nn) return;
    const int i = n % (I.nx + 1);
    const int t = n / (I.nx + 1);
    const int j = t % (I.ny + 1);
    const int k = t / (I.ny + 1);
    const long long gn = I.node_off + n;
    const uint8_t cm = g.clamp[gn];
    const int row = g.srow[gn];
    const double hdt = 0.5 * dt, hdt2 = 0.5 * dt * dt;
    const double minv = g.minv[gn];
    const double* h1 = slot1 >= 0 ? g.hist + I.hist_off + (long long)slot1 * 9 * I.ns : nullptr;
    const double* h2 = slot2 >= 0 ? g.hist + I.hist_off + (long long)slot2 * 9 * I.ns : nullptr;
    const float2* fe = static_cast<const float2*>(g.fe) + I.elem_off;
    // loads first (state, then the element contributions of the three components, summed per
    // component in double-float in the fixed corner order)
    double uc[3], vc[3], ac[3];
    f2 f[3] = {df::make(0.f, 0.f), df::make(0.f, 0.f), df::make(0.f, 0.f)};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const long long d = (long long)c * g.NN + gn;
        uc[c] = ucur[d];
        vc[c] = g.v[d];
        ac[c] = g.a[d];
    }
    if (!predict_only && row < 0 && cm != 7) {
#pragma unroll
        for (int az = 0; az < 2; ++az) {
            const int ke = k - az;
            if (ke < 0 || ke >= I.nz) continue;
#pragma unroll
            for (int ay = 0; ay < 2; ++ay) {
                const int je = j - ay;
                if (je < 0 || je >= I.ny) continue;
#pragma unroll
                for (int ax = 0; ax < 2; ++ax) {
                    const int ie = i - ax;
                    if (ie < 0 || ie >= I.nx) continue;
                    const long long e = ie + (long long)I.nx * (je + I.ny * ke);
                    const int corner = ax + 2 * ay + 4 * az;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float2 v = __ldg(fe + (long long)(corner * 3 + c) * g.NE + e);
                        f[c] = df::add(f[c], df::make(v.x, v.y));
                    }
                }
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const long long d = (long long)c * g.NN + gn;
        double un;
        if (cm & (1 << c)) {
            g.v[d] = 0.0;
            g.a[d] = 0.0;
            un = 0.0;
        } else if (row >= 0) {
            if (!predict_only) {
                g.v[d] = h1[(long long)(3 + c) * I.ns + row];
                g.a[d] = h1[(long long)(6 + c) * I.ns + row];
            }
            un = h2 ? h2[(long long)c * I.ns + row] : 0.0;
        } else {
            double vn = vc[c], an = ac[c];
            if (!predict_only) {
                const double anew = -df::to_double(f[c]) * minv;
                vn = fma(hdt, an + anew, vn);
                an = anew;
                g.v[d] = vn;
                g.a[d] = an;
            }
            un = fma(hdt2, an, fma(dt, vn, uc[c]));
        }
        if (h2) {
            unext[d] = un;
            const f2 s = df::from_double(un * I.invh);
            g.u2[d] = make_float2(s.h, s.l);
        }
    }
}

// double-float copy of u[0] / h (initialisation of the f32x2 force input)
__global__ void __launch_bounds__(kNodeBlock) k_split_u2_b(const FomB g) {
    const int2 b = g.nblk[blockIdx.x];
    const InstFom I = g.inst[b.x];
    const int n = b.y + threadIdx.x;
    if (n >= I.nn) return;
    const long long gn = I.node_off + n;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const df::f2 v = df::from_double(g.u[0][(long long)c * g.NN + gn] * I.invh);
        g.u2[(long long)c * g.NN + gn] = make_float2(v.h, v.l);
    }
}

}  // namespace

cudaError_t launch_force_df_b(const FomB& g, const int* active, const TraceFuse& tr, cudaStream_t s) {
    if (g.n_eblk == 0) return cudaSuccess;
    const int b = g.eblock;
    if (b > 128) return cudaErrorInvalidConfiguration;
    long long items = 0;
    for (int k = 0; k < tr.n; ++k) items += 3LL * tr.c[k].R;
    const int grid = g.n_eblk + (int)((items + b - 1) / b);
    const size_t smem = sizeof(float2) * kDfSlots * b;
    // opt in to more than 48 KB of dynamic shared memory, once per device (the attribute is per device)
    static std::atomic<unsigned long long> attr_set{0};
    int dev = 0;
    cudaError_t ed = cudaGetDevice(&dev);
    if (ed != cudaSuccess) return ed;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(attr_set.load() & bit)) {
        const int max_bytes = (int)(sizeof(float2) * kDfSlots * 128);
        cudaError_t e1 = cudaFuncSetAttribute(k_force_df2_b<OSAM_NEO_HOOKEAN>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaError_t e2 = cudaFuncSetAttribute(k_force_df2_b<OSAM_LINEAR_ELASTIC>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaError_t e3 = cudaFuncSetAttribute(k_force_df2_b<OSAM_SAINT_VENANT_KIRCHHOFF>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        if (e1 != cudaSuccess) return e1;
        if (e2 != cudaSuccess) return e2;
        if (e3 != cudaSuccess) return e3;
        attr_set.fetch_or(bit);
    }
    if (g.material == OSAM_NEO_HOOKEAN) k_force_df2_b<OSAM_NEO_HOOKEAN><<<grid, b, smem, s>>>(g, active, tr);
    else if (g.material == OSAM_SAINT_VENANT_KIRCHHOFF) k_force_df2_b<OSAM_SAINT_VENANT_KIRCHHOFF><<<grid, b, smem, s>>>(g, active, tr);
    else k_force_df2_b<OSAM_LINEAR_ELASTIC><<<grid, b, smem, s>>>(g, active, tr);
    return cudaGetLastError();
}

cudaError_t launch_node_df_b(const FomB& g, const int* active, int slot1, int slot2, int predict_only,
                             const double* ucur, double* unext, double dt, cudaStream_t s) {
    k_node_df_b<<<g.n_nblk, kNodeBlock, 0, s>>>(g, active, slot1, slot2, predict_only, ucur, unext, dt);
    return cudaGetLastError();
}

cudaError_t launch_split_u2_b(const FomB& g, cudaStream_t s) {
    k_split_u2_b<<<g.n_nblk, kNodeBlock, 0, s>>>(g);
    return cudaGetLastError();
}

}  // namespace osam
