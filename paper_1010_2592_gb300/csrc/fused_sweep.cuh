// Fused FP32 sweeps of the double-pass solver (Sec. 2): the BiCG vector
// updates of a sub-step are folded into the hop that consumes them, and the
// MR Gram matrix into the epilogue of the last hop of the outer iteration.
//
// One BiCG sub-step j of BiCGstab(l) (pass 1) is four sweeps:
//   F1  tmp = g5 D (r_j - beta u_j); the updated u_j is written to its
//       alternate buffer; u_i <- r_i - beta u_i (i < j) at the sweep's own sites
//   F2  u_{j+1} = c g5 D tmp; partials of <rt, u_{j+1}>; alpha in the last block
//   F3  tmp = g5 D (r_j - alpha u_{j+1}); the updated r_j to its alternate
//       buffer; r_i <- r_i - alpha u_{i+1} (i < j) at the own sites; the
//       pseudo-double-pass store of the occurrences r_i (i <= j) before the
//       update, or in pass 2 their weighted sum into y; block 0 runs the shift
//       part of the sub-step (the zeta recurrences)
//   F4  r_{j+1} = c g5 D tmp; partials of <rt, r_{j+1}> and the next beta, or
//       after the last sub-step the Gram matrix <r_i, r_k> (i <= k <= l) and
//       the MR coefficients gamma in the last block.
// The updated vector is formed at every stencil point from the two stored
// ones (a + c b with one fused multiply-add per component, the same operation
// the unfused update kernel performs), so every read of it sees the value its
// owner writes.  The owner writes it to a second buffer because other threads
// of the same sweep still read the old one: within an outer iteration u_j and
// r_j (j < l) move to their alternate buffers, the MR kernel writes r_0, u_0
// back to the home buffers, and r_{j+1}, u_{j+1} are regenerated there, so
// every outer iteration starts from the same buffers and its launches are
// iteration-independent (CUDA-graph replay).
#pragma once

#include "solver_kernels.cuh"

namespace fa {

// in = a + c b formed as it is read (FP32 [6][V] chunks, c complex)
struct AxpyView32 {
    const float4* a;
    const float4* b;
    cx<float> c;
    int V;
    __device__ __forceinline__ void load(int s, cx<float> v[12]) const {
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const float4 x = __ldg(a + (size_t)q * V + s), y = __ldg(b + (size_t)q * V + s);
            v[2 * q] = cfma(c, cx<float>{y.x, y.y}, cx<float>{x.x, x.y});
            v[2 * q + 1] = cfma(c, cx<float>{y.z, y.w}, cx<float>{x.z, x.w});
        }
    }
};

// Arguments of the first hop of A (F1 / F3), passed by value (parameter space).
struct FusedHop1 {
    Geom g;
    LinkView<float> U;
    const float4* a;                 // stencil input a + c b (r_j and u_j, or r_j and u_{j+1})
    const float4* b;
    float4* tmp;                     // g5 D (a + c b)
    float4* upd;                     // the updated vector at the own sites (alternate buffer)
    float4* cdst[kMaxEll];           // own-site updates dst_i <- a_i + c b_i, i < j
    const float4* ca[kMaxEll];
    const float4* cb[kMaxEll];
    const float4* u0;                // reliable updates: u_0 after this sub-step's update (x += alpha u_0)
    float cdiag, chop, ef, eb, bc;   // the first hop of A: scale 1
    int j;                           // BiCG sub-step
};

// Arguments of the second hop of A (F2 / F4).
struct FusedHop2 {
    Geom g;
    LinkView<float> U;
    const float4* in;                // tmp
    float4* out;                     // u_{j+1} or r_{j+1} (home buffer)
    const float4* rt;                // shadow vector (inner products)
    double2* part;                   // reduction partials
    const float4* gram[kMaxEll];     // r_0 .. r_{l-1} after their updates (Gram epilogue)
    float cdiag, chop, ef, eb, bc;   // scale c
};

// F1 (KIND 0, c = -beta_j) and F3 (KIND 1, c = -alpha_j).  XS: block 0 runs the
// shift part of sub-step j (pass 1 of the double-pass forms).  ACC: pass 2,
// y += sum_i coef r_i(before the update), i <= j.
template <int L, int KIND, bool XS, bool ACC, int NT, int MB>
__global__ void __launch_bounds__(NT, MB)
k_fhop1(FusedHop1 A, const SolverDev* __restrict__ ds, int pass2) {
    dep_sync();
    const SolverDev& d = ds[0];
    if (sys_idle(d, pass2)) return;
    const int j = A.j;
    if (XS && blockIdx.x == 0) {
        sc_alpha_shifts(d, j);
        return;
    }
    const int s = (int)(blockIdx.x - (XS ? 1u : 0u)) * NT + (int)threadIdx.x;
    if (s >= A.g.V) return;
    const int m = d.st->m;
    const int V = A.g.V;
    const cx<float> c = negcx<float>(KIND == 0 ? d.rec_beta[m * L + j] : d.rec_alpha[m * L + j]);
    {
        const AxpyView32 in{A.a, A.b, c, V};
        cx<float> p[12], pin[12];
        hop_site<float, false, true, true>(A.g, A.U, in, s, A.cdiag, A.chop, A.ef, A.eb, A.bc, p, pin);
        SpinorView<float>{A.tmp, V}.store(s, p);
        SpinorView<float>{A.upd, V}.store(s, pin);
    }
    // own-site work, chunk by chunk
    float4* store = nullptr;
    if (KIND == 1 && !ACC && !pass2) store = store_at<float>(d, m);
    const size_t vs = (size_t)6 * V;
    const size_t cf0 = (size_t)m * nc_slots(L);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        cx<float> t[2] = {czero<float>(), czero<float>()};
        // compile-time indices into the parameter arrays (no local copy of them)
#pragma unroll
        for (int i = 0; i < L; ++i) {
            if (i >= j) break;
            const float4 x = __ldg(A.ca[i] + (size_t)q * V + s), y = __ldg(A.cb[i] + (size_t)q * V + s);
            if (KIND == 1) {
                // x is r_i before this sub-step's update (the occurrence r_old_i)
                if (store != nullptr) store[slot_old(j, i) * vs + (size_t)q * V + s] = x;
                if (ACC) {
                    const cx<float> w = weight<float>(d.coef, d.coef4, cf0 + slot_old(j, i));
                    t[0] = cfma(w, cx<float>{x.x, x.y}, t[0]);
                    t[1] = cfma(w, cx<float>{x.z, x.w}, t[1]);
                }
            }
            const cx<float> n0 = cfma(c, cx<float>{y.x, y.y}, cx<float>{x.x, x.y});
            const cx<float> n1 = cfma(c, cx<float>{y.z, y.w}, cx<float>{x.z, x.w});
            A.cdst[i][(size_t)q * V + s] = make_float4(n0.r, n0.i, n1.r, n1.i);
        }
        if (KIND == 1) {
            // the occurrence r_old_j: r_j before the update, at the own site
            const float4 x = __ldg(A.a + (size_t)q * V + s);
            if (store != nullptr) store[slot_old(j, j) * vs + (size_t)q * V + s] = x;
            if (ACC) {
                const cx<float> w = weight<float>(d.coef, d.coef4, cf0 + slot_old(j, j));
                t[0] = cfma(w, cx<float>{x.x, x.y}, t[0]);
                t[1] = cfma(w, cx<float>{x.z, x.w}, t[1]);
                acc_y<float>(d.y, q, V, s, t);
            }
            if (d.x64 != nullptr) {
                Ch<float> u;
                const float4 uu = __ldg(A.u0 + (size_t)q * V + s);
                u.c[0] = {uu.x, uu.y};
                u.c[1] = {uu.z, uu.w};
                acc_x<float>(d.x64, q, V, s, d.rec_alpha[m * L + j], u);
            }
        }
    }
}

// F2 / F4.  RED 0: none; 1: <rt, out> partials and `step` in the last block;
// 2: Gram partials <r_i, r_k> (i <= k <= L, r_L = out) and the MR coefficients
// (sc_mr_seed) in the last block.
template <int L, int RED, int NT, int MB>
__global__ void __launch_bounds__(NT, MB)
k_fhop2(FusedHop2 A, const SolverDev* __restrict__ ds, int pass2, ScalarStep step) {
    dep_sync();
    const SolverDev& d = ds[0];
    if (sys_idle(d, pass2)) return;
    const int s = (int)blockIdx.x * NT + (int)threadIdx.x;
    const int V = A.g.V;
    constexpr int NR = RED == 2 ? n_gram(L) : 1;
    cx<float> red[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) red[k] = czero<float>();
    if (s < V) {
        cx<float> p[12];
        hop_site<float, false, true>(A.g, A.U, SpinorView<float>{const_cast<float4*>(A.in), V}, s, A.cdiag, A.chop,
                                     A.ef, A.eb, A.bc, p);
        SpinorView<float>{A.out, V}.store(s, p);
        if constexpr (RED == 1) {
            cx<float> q[12];
            SpinorView<float>{const_cast<float4*>(A.rt), V}.load(s, q);
#pragma unroll
            for (int k = 0; k < 12; ++k) red[0] = cjfma(q[k], p[k], red[0]);
        } else if constexpr (RED == 2) {
            // the same (i, k) order as the unfused Gram kernel, chunk by chunk
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                cx<float> v[L + 1][2];
#pragma unroll
                for (int i = 0; i < L; ++i) {
                    const float4 x = __ldg(A.gram[i] + (size_t)q * V + s);
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
    }
    if constexpr (RED == 1) {
        block_reduce_store<1, float, NT>(red, A.part, 0, blockIdx.x);
        run_step<true>(d, step, gridDim.x);
    } else if constexpr (RED == 2) {
        block_reduce_store<NR, float, NT>(red, A.part, gridDim.x, blockIdx.x);
        if (last_block(d.st)) sc_mr_seed<L, true>(d, gridDim.x);
    }
}

}  // namespace fa
