// The MR Gram matrix of the double-pass solver (Sec. 2) formed in the epilogue
// of the last FP32 D_w sweep of an outer iteration.
//
// The last sweep of BiCG sub-step l-1 produces r_l = c g5 D tmp; the MR step
// then needs <r_i, r_k> for 0 <= i <= k <= l.  Instead of a kernel of its own
// that reads r_0..r_l again, the sweep that holds r_l in registers reads
// r_0..r_{l-1} at its own sites and stores the per-block partials; its last
// block solves for the MR coefficients gamma (sc_mr_seed).  No stencil read
// changes, so the sweep keeps its neighbour traffic; one launch and one pass
// over r_l less per outer iteration.
//
// Measured on GB300, 16^3 x 32: folding the BiCG vector updates u_i <- r_i -
// beta u_i and r_i <- r_i - alpha u_{i+1} into the sweeps as well (forming the
// updated vector at each of the nine stencil points from the two stored ones)
// made the outer iteration slower (254 against 219 us), because it doubles the
// neighbour loads of a latency-bound stencil; those updates keep their own
// kernels.
#pragma once

#include "solver_kernels.cuh"

namespace fa {

// Arguments of the Gram sweep, passed by value (parameter space).
struct GramHop {
    Geom g;
    LinkView<float> U;
    const float4* in;                // tmp = g5 D r_{l-1}
    float4* out;                     // r_l
    double2* part;                   // reduction partials, n_gram(l) slots of gridDim.x
    const float4* r[kMaxEll];        // r_0 .. r_{l-1}
    float cdiag, chop, ef, eb, bc;   // the second hop of A: scale c
};

// r_l = c g5 D tmp and the partials of <r_i, r_k> (i <= k <= L) in the order of
// the Gram kernel, then the MR coefficients in the last block.
template <int L, int NT, int MB>
__global__ void __launch_bounds__(NT, MB)
k_hop_gram(GramHop A, const SolverDev* __restrict__ ds) {
    dep_sync();
    const TraceScope trace_(trace_kind<float>(FA_TK_HOP_GRAM));
    const SolverDev& d = ds[0];
    if (sys_idle(d, 0)) return;
    const int s = (int)blockIdx.x * NT + (int)threadIdx.x;
    const int V = A.g.V;
    constexpr int NG = n_gram(L);
    cx<float> red[NG];
#pragma unroll
    for (int k = 0; k < NG; ++k) red[k] = czero<float>();
    if (s < V) {
        cx<float> p[12];
        hop_site<float, false, true>(A.g, A.U, SpinorView<float>{const_cast<float4*>(A.in), V}, s, A.cdiag, A.chop,
                                     A.ef, A.eb, A.bc, p);
        SpinorView<float>{A.out, V}.store(s, p);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            cx<float> v[L + 1][2];
#pragma unroll
            for (int i = 0; i < L; ++i) {
                const float4 x = __ldg(A.r[i] + (size_t)q * V + s);
                v[i][0] = {x.x, x.y};
                v[i][1] = {x.z, x.w};
            }
            v[L][0] = p[2 * q];
            v[L][1] = p[2 * q + 1];
            int gi = 0;
#pragma unroll
            for (int i = 0; i <= L; ++i)
#pragma unroll
                for (int k = i; k <= L; ++k) {
#pragma unroll
                    for (int w = 0; w < 2; ++w) red[gi] = cjfma(v[i][w], v[k][w], red[gi]);
                    ++gi;
                }
        }
    }
    block_reduce_store<NG, float, NT>(red, A.part, gridDim.x, blockIdx.x);
    const int lb = last_block(d.st, gridDim.x);
    if (lb != LB_NONE) sc_mr_seed<L, true>(d, gridDim.x, lb == LB_WARM);
}

}  // namespace fa
