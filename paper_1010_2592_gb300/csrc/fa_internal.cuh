// Internal definitions shared by the CUDA translation units of libfapath.
//
// Internal layouts (structure of arrays, one thread per lattice site):
//   FP64 spinor  double2 [12][V]        component k = 3*spin + colour
//   FP32 spinor  float4  [6][V]         chunk q holds components 2q, 2q+1
//   FP64 links   double2 [4][9][V]      element 3*row + col of U_mu(x)
//   FP32 links   float4  [4][3][V]      rows 0-1 (6 complex); row 2 rebuilt
// Site index s = x + X*(y + Y*(z + Z*t)), as in the canonical layout.
#pragma once

#include <type_traits>

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

#include "fapath.h"

namespace fa {

constexpr int kMaxEll = 8;
constexpr int kMaxShifts = 64;
constexpr int kThreads = 256;          // block size of all site kernels
constexpr int kScalarThreads = 256;    // block size of the single-block kernels (power-iteration norm)

struct Geom {
    int X, Y, Z, T;
    int V;
};

// Programmatic dependent launch.  A kernel launched with programmatic stream
// serialization may be placed on the SMs while its predecessor in the stream
// is still running; it must not touch global memory before `griddepcontrol.wait`
// returns, which happens once the predecessor grid has completed and its writes
// are visible.  `launch_dependents` then lets the successor start its own launch.
// For an ordinary launch both instructions return at once.  Every kernel that
// the solver may launch this way calls this first.
__device__ __forceinline__ void dep_sync() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ------------------------------------------------------------------ complex
template <typename R> struct cx { R r, i; };

__device__ __forceinline__ float fmaR(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmaR(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mulR(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mulR(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float addR(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double addR(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float subR(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double subR(double a, double b) { return __dsub_rn(a, b); }

// ------------------------------------------------------------------ double-float
// A "double-float" value is the unevaluated sum hi + lo of two FP32 numbers
// with |lo| <= ulp(hi)/2: about 44-48 significant bits computed on the FP32
// pipes (GB300 runs FP32 at many times its FP64 rate).  Sums use Knuth's
// TwoSum (the exact rounding error of an addition) and products Dekker's
// TwoProduct in its FMA form (e = fma(a, b, -a*b) is exact); the result is
// renormalised with Fast-TwoSum.  Additions use the short form (one TwoSum on
// the high parts): the error is about 2^-44 of the larger operand.
struct df {
    float hi, lo;
    df() = default;
    __host__ __device__ constexpr df(float h, float l = 0.0f) : hi(h), lo(l) {}
};

__device__ __forceinline__ df fast_two_sum(float a, float b) {   // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ df addR(df a, df b) {
    const df s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df subR(df a, df b) { return addR(a, df(-b.hi, -b.lo)); }
__device__ __forceinline__ df mulR(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ df fmaR(df a, df b, df c) { return addR(mulR(a, b), c); }
__device__ __forceinline__ df operator-(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df operator+(df a, df b) { return addR(a, b); }
__device__ __forceinline__ df operator-(df a, df b) { return subR(a, b); }
// sign factors of the projectors (exact)
__device__ __forceinline__ df operator*(int s, df a) { return {(float)s * a.hi, (float)s * a.lo}; }

// conversions between the working precisions and FP64
__device__ __forceinline__ double todbl(float x) { return (double)x; }
__device__ __forceinline__ double todbl(double x) { return x; }
__device__ __forceinline__ double todbl(df x) { return __dadd_rn((double)x.hi, (double)x.lo); }
template <typename R> __device__ __forceinline__ R fromdbl(double x) { return (R)x; }
template <> __device__ __forceinline__ df fromdbl<df>(double x) {
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(__dsub_rn(x, (double)h))};
}
// the same conversions on the host (kernel arguments)
template <typename R> inline R host_cvt(double x) { return (R)x; }
template <> inline df host_cvt<df>(double x) {
    const float h = (float)x;
    return df(h, (float)(x - (double)h));
}

template <typename R> __device__ __forceinline__ cx<R> czero() { return {R(0), R(0)}; }
template <typename R> __device__ __forceinline__ cx<R> cadd(cx<R> a, cx<R> b) { return {addR(a.r, b.r), addR(a.i, b.i)}; }
template <typename R> __device__ __forceinline__ cx<R> csub(cx<R> a, cx<R> b) { return {subR(a.r, b.r), subR(a.i, b.i)}; }
// acc + a*b
template <typename R> __device__ __forceinline__ cx<R> cfma(cx<R> a, cx<R> b, cx<R> acc) {
    acc.r = fmaR(a.r, b.r, acc.r);
    acc.r = fmaR(-a.i, b.i, acc.r);
    acc.i = fmaR(a.r, b.i, acc.i);
    acc.i = fmaR(a.i, b.r, acc.i);
    return acc;
}
// acc + conj(a)*b
template <typename R> __device__ __forceinline__ cx<R> cjfma(cx<R> a, cx<R> b, cx<R> acc) {
    acc.r = fmaR(a.r, b.r, acc.r);
    acc.r = fmaR(a.i, b.i, acc.r);
    acc.i = fmaR(a.r, b.i, acc.i);
    acc.i = fmaR(-a.i, b.r, acc.i);
    return acc;
}
template <typename R> __device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
    cx<R> t;
    t.r = fmaR(-a.i, b.i, mulR(a.r, b.r));
    t.i = fmaR(a.i, b.r, mulR(a.r, b.i));
    return t;
}
template <typename R> __device__ __forceinline__ cx<R> cscale(R s, cx<R> a) { return {mulR(s, a.r), mulR(s, a.i)}; }
// acc + s*a, s real
template <typename R> __device__ __forceinline__ cx<R> crfma(R s, cx<R> a, cx<R> acc) {
    return {fmaR(s, a.r, acc.r), fmaR(s, a.i, acc.i)};
}

// host/device double complex helpers for scalar work (FP64, run by one thread)
struct dcx { double r, i; };
__host__ __device__ __forceinline__ dcx mk(double r, double i = 0.0) { return {r, i}; }
__host__ __device__ __forceinline__ dcx operator+(dcx a, dcx b) { return {a.r + b.r, a.i + b.i}; }
__host__ __device__ __forceinline__ dcx operator-(dcx a, dcx b) { return {a.r - b.r, a.i - b.i}; }
__host__ __device__ __forceinline__ dcx operator-(dcx a) { return {-a.r, -a.i}; }
__host__ __device__ __forceinline__ dcx operator*(dcx a, dcx b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
__host__ __device__ __forceinline__ dcx operator*(double s, dcx a) { return {s * a.r, s * a.i}; }
__host__ __device__ __forceinline__ dcx conjd(dcx a) { return {a.r, -a.i}; }
__host__ __device__ __forceinline__ double abs2(dcx a) { return a.r * a.r + a.i * a.i; }
// a / b using the library division on the real parts
__host__ __device__ __forceinline__ dcx operator/(dcx a, dcx b) {
    double d = b.r * b.r + b.i * b.i;
    return {(a.r * b.r + a.i * b.i) / d, (a.i * b.r - a.r * b.i) / d};
}
__host__ __device__ __forceinline__ bool finite(dcx a) { return isfinite(a.r) && isfinite(a.i); }
__device__ __forceinline__ dcx ld(const double2& v) { return {v.x, v.y}; }
__device__ __forceinline__ double2 pk(dcx v) { return make_double2(v.r, v.i); }

// ------------------------------------------------------------------ spinor views
template <typename R> struct SpinorView;

template <> struct SpinorView<double> {
    double2* p;
    int V;
    __device__ __forceinline__ void load(int s, cx<double> v[12]) const {
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            double2 t = __ldg(p + (size_t)k * V + s);
            v[k] = {t.x, t.y};
        }
    }
    __device__ __forceinline__ void store(int s, const cx<double> v[12]) const {
#pragma unroll
        for (int k = 0; k < 12; ++k) p[(size_t)k * V + s] = make_double2(v[k].r, v[k].i);
    }
    __device__ __forceinline__ cx<double> ld1(int s, int k) const {
        const double2 t = __ldg(p + (size_t)k * V + s);
        return {t.x, t.y};
    }
    __device__ __forceinline__ void st1(int s, int k, cx<double> v) const {
        p[(size_t)k * V + s] = make_double2(v.r, v.i);
    }
};

template <> struct SpinorView<float> {
    float4* p;
    int V;
    __device__ __forceinline__ void load(int s, cx<float> v[12]) const {
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            float4 t = __ldg(p + (size_t)q * V + s);
            v[2 * q] = {t.x, t.y};
            v[2 * q + 1] = {t.z, t.w};
        }
    }
    __device__ __forceinline__ void store(int s, const cx<float> v[12]) const {
#pragma unroll
        for (int q = 0; q < 6; ++q)
            p[(size_t)q * V + s] = make_float4(v[2 * q].r, v[2 * q].i, v[2 * q + 1].r, v[2 * q + 1].i);
    }
};

template <> struct SpinorView<df> {
    float4* p;
    int V;
    __device__ __forceinline__ void load(int s, cx<df> v[12]) const {
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            float4 t = __ldg(p + (size_t)k * V + s);
            v[k] = {df(t.x, t.y), df(t.z, t.w)};
        }
    }
    __device__ __forceinline__ void store(int s, const cx<df> v[12]) const {
#pragma unroll
        for (int k = 0; k < 12; ++k) p[(size_t)k * V + s] = make_float4(v[k].r.hi, v[k].r.lo, v[k].i.hi, v[k].i.lo);
    }
    __device__ __forceinline__ cx<df> ld1(int s, int k) const {
        const float4 t = __ldg(p + (size_t)k * V + s);
        return {df(t.x, t.y), df(t.z, t.w)};
    }
    __device__ __forceinline__ void st1(int s, int k, cx<df> v) const {
        p[(size_t)k * V + s] = make_float4(v.r.hi, v.r.lo, v.i.hi, v.i.lo);
    }
};

// bytes of one internal spinor
template <typename R> constexpr size_t spinor_bytes(int V) { return (size_t)V * 12 * 2 * sizeof(R); }

// ------------------------------------------------------------------ link views
template <typename R> struct LinkView;

template <> struct LinkView<double> {
    const double2* p;
    int V;
    __device__ __forceinline__ void load(int mu, int s, cx<double> U[3][3]) const {
        const double2* b = p + (size_t)mu * 9 * V + s;
#pragma unroll
        for (int e = 0; e < 9; ++e) {
            double2 t = __ldg(b + (size_t)e * V);
            U[e / 3][e % 3] = {t.x, t.y};
        }
    }
    // element (row, col) = e / 3, e % 3
    __device__ __forceinline__ cx<double> ld1(int mu, int s, int e) const {
        const double2 t = __ldg(p + ((size_t)mu * 9 + e) * V + s);
        return {t.x, t.y};
    }
};

template <> struct LinkView<float> {
    const float4* p;
    int V;
    __device__ __forceinline__ void load(int mu, int s, cx<float> U[3][3]) const {
        const float4* b = p + (size_t)mu * 3 * V + s;
        float4 a0 = __ldg(b), a1 = __ldg(b + V), a2 = __ldg(b + 2 * (size_t)V);
        U[0][0] = {a0.x, a0.y}; U[0][1] = {a0.z, a0.w}; U[0][2] = {a1.x, a1.y};
        U[1][0] = {a1.z, a1.w}; U[1][1] = {a2.x, a2.y}; U[1][2] = {a2.z, a2.w};
        // row 2 = conj(row 0 x row 1): unitary rows with det 1
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
            cx<float> t = cmul(U[0][c1], U[1][c2]);
            t = cfma(cx<float>{-U[0][c2].r, -U[0][c2].i}, U[1][c1], t);
            U[2][c] = {t.r, -t.i};
        }
    }
};

template <> struct LinkView<df> {
    const float4* p;
    int V;
    __device__ __forceinline__ void load(int mu, int s, cx<df> U[3][3]) const {
        const float4* b = p + (size_t)mu * 9 * V + s;
#pragma unroll
        for (int e = 0; e < 9; ++e) {
            float4 t = __ldg(b + (size_t)e * V);
            U[e / 3][e % 3] = {df(t.x, t.y), df(t.z, t.w)};
        }
    }
    __device__ __forceinline__ cx<df> ld1(int mu, int s, int e) const {
        const float4 t = __ldg(p + ((size_t)mu * 9 + e) * V + s);
        return {df(t.x, t.y), df(t.z, t.w)};
    }
};

// ------------------------------------------------------------------ block reduction
// Sum K complex values over the block; thread 0 writes them to
// out[k*stride + bidx].  FP64 values are summed in FP64 and stored as double2.
// FP32 values are summed in FP32 within a warp, double-float values in
// double-float; both then in double-float across warps and stored as an FP32
// pair per part (float4: re.hi, re.lo, im.hi, im.lo) in the same 16 bytes, so
// that no FP64 instruction is spent (they are scarce on this part).
// Deterministic for a fixed launch shape.
__device__ __forceinline__ df shfl_down_df(df a, int o) {
    return df(__shfl_down_sync(0xffffffffu, a.hi, o), __shfl_down_sync(0xffffffffu, a.lo, o));
}

template <int K, typename R, int NT = kThreads>
__device__ __forceinline__ void block_reduce_store(cx<R> (&v)[K], double2* out, int stride, int bidx) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (sizeof(R) == 8 && !std::is_same<R, df>::value) {
        __shared__ double2 sh[K][NW];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double a = v[k].r, b = v[k].i;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a += __shfl_down_sync(0xffffffffu, a, o);
                b += __shfl_down_sync(0xffffffffu, b, o);
            }
            if (lane == 0) sh[k][warp] = make_double2(a, b);
        }
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                double a = 0.0, b = 0.0;
                if (lane < NW) { a = sh[k][lane].x; b = sh[k][lane].y; }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    a += __shfl_down_sync(0xffffffffu, a, o);
                    b += __shfl_down_sync(0xffffffffu, b, o);
                }
                if (lane == 0) out[(size_t)k * stride + bidx] = make_double2(a, b);
            }
        }
    } else {
        __shared__ float4 sh[K][NW];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if constexpr (std::is_same<R, float>::value) {
                float a = v[k].r, b = v[k].i;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    a += __shfl_down_sync(0xffffffffu, a, o);
                    b += __shfl_down_sync(0xffffffffu, b, o);
                }
                if (lane == 0) sh[k][warp] = make_float4(a, 0.0f, b, 0.0f);
            } else {
                df a = v[k].r, b = v[k].i;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    a = addR(a, shfl_down_df(a, o));
                    b = addR(b, shfl_down_df(b, o));
                }
                if (lane == 0) sh[k][warp] = make_float4(a.hi, a.lo, b.hi, b.lo);
            }
        }
        __syncthreads();
        if (warp == 0) {
            constexpr int TOP = NW > 16 ? 16 : NW > 8 ? 8 : NW > 4 ? 4 : NW > 2 ? 2 : 1;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                df a(0.0f), b(0.0f);
                if (lane < NW) {
                    const float4 t = sh[k][lane];
                    a = df(t.x, t.y);
                    b = df(t.z, t.w);
                }
#pragma unroll
                for (int o = TOP; o > 0; o >>= 1) {
                    a = addR(a, shfl_down_df(a, o));
                    b = addR(b, shfl_down_df(b, o));
                }
                if (lane == 0)
                    reinterpret_cast<float4*>(out)[(size_t)k * stride + bidx] = make_float4(a.hi, a.lo, b.hi, b.lo);
            }
        }
    }
}
template <int K, typename R>
__device__ __forceinline__ void block_reduce_store(cx<R> (&v)[K], double2* out, int stride) {
    block_reduce_store<K, R>(v, out, stride, blockIdx.x);
}

// ------------------------------------------------------------------ operator params
struct OpParams {
    double diag;      // 4 + m
    double ef, eb;    // e^{+mu}, e^{-mu}
    double t_bc;      // time boundary sign
    double scale;     // c
};

// ------------------------------------------------------------------ host-side API of the kernels
// Records "what: <CUDA error>" as the library's last error and returns FA_ECUDA.
int cuda_fail(cudaError_t e, const char* what);
// FA_OK after a launch, else the launch error recorded by cuda_fail.
inline int launch_status(const char* what) {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FA_OK : cuda_fail(e, what);
}

// Hop (one D_w sweep): out = scale * G5OUT * (diag*in' - 1/2 sum hops(in')),
// in' = G5IN ? gamma_5 in : in, time weights from `mu_sign` * mu.
// When dot_with != nullptr, per-block partials of <dot_with, out> are written
// to partials[blockIdx] (nblk = ceil(V/kThreads) of them).
int launch_hop_f64(const Geom& g, const double2* links, const double2* in, double2* out,
                   double diag, double ef, double eb, double t_bc, double scale,
                   bool g5in, bool g5out, const double2* dot_with, double2* partials,
                   const int* done, cudaStream_t st);
// shape: 0 narrow when the lattice fits one wave of it, 1 wide (kThreads x
// FA_HOP_MINB per SM), 2 narrow (kHopNarrowThreads x kHopNarrowBlocks per SM)
int launch_hop_f32(const Geom& g, const float4* links, const float4* in, float4* out,
                   double diag, double ef, double eb, double t_bc, double scale,
                   bool g5in, bool g5out, const float4* dot_with, double2* partials,
                   const int* done, cudaStream_t st, int shape = 0);

int launch_hop_df(const Geom& g, const float4* links, const float4* in, float4* out,
                  double diag, double ef, double eb, double t_bc, double scale,
                  bool g5in, bool g5out, const float4* dot_with, double2* partials,
                  const int* done, cudaStream_t st);

// canonical (interleaved complex128 AoS) <-> internal layouts
int launch_pack_spinor_f64(const Geom& g, const double* canon, double2* out, cudaStream_t st);
int launch_unpack_spinor_f64(const Geom& g, const double2* in, double* canon, cudaStream_t st);
int launch_pack_spinor_f32(const Geom& g, const double* canon, float4* out, cudaStream_t st);
int launch_unpack_spinor_f32(const Geom& g, const float4* in, double* canon, cudaStream_t st);
int launch_pack_links(const Geom& g, const double* canon, double2* l64, float4* l32, float4* ldf, cudaStream_t st);
// SMs of the current device; whether an FP32 sweep of V sites uses the narrow
// launch shape (kHopNarrowThreads x kHopNarrowBlocks per SM, one wave)
int sm_count();
bool hop_narrow(int V);
// the narrow shape for a sweep of V sites under launch shape `shape`
inline bool hop_use_narrow(int shape, int V) { return shape == 2 || (shape == 0 && hop_narrow(V)); }
int launch_convert_f64_to_f32(const Geom& g, const double2* in, float4* out, cudaStream_t st);
// double-float spinors: [12][V] float4 = (re.hi, re.lo, im.hi, im.lo)
int launch_pack_spinor_df(const Geom& g, const double* canon, float4* out, cudaStream_t st);
int launch_unpack_spinor_df(const Geom& g, const float4* in, double* canon, cudaStream_t st);
int launch_convert_df_to_f32(const Geom& g, const float4* in, float4* out, cudaStream_t st);

// adjoint link force of <a1, D b1> + <a2, D b2> (a1 enters as gamma_5 a1), scaled by w,
// added to the canonical gradient G; per-block partials of the mu-derivative.
int launch_force(const Geom& g, const double2* links, const double2* a1, const double2* b1, const double2* a2,
                 const double2* b2, double* G_canon, double w, double ef, double eb, double t_bc,
                 double2* partials, cudaStream_t st);

inline int nblocks(int V) { return (V + kThreads - 1) / kThreads; }

}  // namespace fa
