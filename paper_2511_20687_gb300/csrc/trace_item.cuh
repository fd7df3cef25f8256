// Overlap trace Pi(u, v, a) at a neighbour's Schwarz nodes (Sec. 3, pointwise trilinear projector),
// shared by the stand-alone trace kernel and the trace blocks appended to an internal-force grid.
#pragma once

#include <cuda_runtime.h>

#include "osam_internal.h"

namespace osam {
namespace trace {

// one work item of the overlap trace: row gr = t / 3, component t % 3 of u, v and a interpolated at
// the row's donor nodes with the trilinear weights, recorded at history slot `slot`
__device__ __forceinline__ void trace_item(const CplB& c, const int* __restrict__ active, const FomB& src,
                                           const double* u, int slot, int t) {
    const int gr = t / 3, cc = t % 3;
    const int inst = c.rinst[gr];
    if (active && !active[inst]) return;
    const int li = gr - c.row_first[inst], nr = c.nrow[inst];
    double su = 0.0, sv = 0.0, sa = 0.0;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const double w = c.dw[8 * gr + b];
        const long long d = (long long)cc * src.NN + c.dnode[8 * gr + b];
        su = fma(w, u[d], su);
        sv = fma(w, src.v[d], sv);
        sa = fma(w, src.a[d], sa);
    }
    double* r = c.rec + c.rec_off[inst] + (long long)slot * 9 * nr;
    r[(long long)(0 + cc) * nr + li] = su;
    r[(long long)(3 + cc) * nr + li] = sv;
    r[(long long)(6 + cc) * nr + li] = sa;
}

// the trace blocks appended to a force grid (block tb counted from the first trace block)
__device__ __forceinline__ void fused_trace_block(const TraceFuse& tr, const int* __restrict__ active,
                                                  const FomB& g, int tb) {
    int t = tb * (int)blockDim.x + (int)threadIdx.x;
#pragma unroll
    for (int k = 0; k < kMaxFusedTraces; ++k) {
        if (k >= tr.n) return;
        if (t < 3 * tr.c[k].R) {
            trace_item(tr.c[k], active, g, tr.u, tr.slot, t);
            return;
        }
        t -= 3 * tr.c[k].R;
    }
}

}  // namespace trace
}  // namespace osam
