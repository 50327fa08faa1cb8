// Kernel timeline tracing of the solver's kernels (fa_trace_start / fa_trace_stop).
//
// While tracing is on, thread 0 of every block of a traced kernel reads the
// GPU's global nanosecond timer (%globaltimer) when the block enters the kernel
// body and again when thread 0 leaves it, and appends one record (entry, exit,
// kernel, block, SM, grid size) to a ring of its SM.  A launch then spans from
// the earliest entry to the latest exit of its blocks; the exit of the last
// block includes the scalar step it runs.  Unlike CUDA events, the records need
// no work between launches, so they time the kernels of a replayed CUDA graph
// as they run in the solve.
//
// Cost when tracing is off: one timer read per block and one constant-cache
// load of the tracer state at exit.  When on: one atomic increment of a per-SM
// counter and one 32-byte store per block.
#pragma once

#include "fa_internal.cuh"

namespace fa {

struct TraceRec {                 // the layout of fa_trace_record
    unsigned long long t0, t1;
    int kind, block, sm, grid;
};
static_assert(sizeof(TraceRec) == sizeof(fa_trace_record), "trace record layout");

struct TraceState {
    TraceRec* rec;                // nullptr: tracing off
    unsigned* pos;                // [nsm] records appended per SM (counts past per_sm)
    unsigned* dropped;            // records that did not fit their SM's ring
    unsigned per_sm;              // ring length per SM
    unsigned nsm;
};
// One per module (only this translation unit's kernels are traced); in
// constant memory, so the check at block exit is a broadcast from the constant
// cache.  Changed only while no traced kernel runs (the host synchronises the
// device first).
static __constant__ TraceState g_trace;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// kernel identifier: FA_TK_* | (working precision << 8) | (variant bit << 10)
template <typename R> constexpr int trace_prec() {
    return std::is_same<R, double>::value ? 0 : (std::is_same<R, float>::value ? 1 : 2);
}
template <typename R> constexpr int trace_kind(int id, bool variant = false) {
    return id | (trace_prec<R>() << 8) | ((variant ? 1 : 0) << 10);
}

struct TraceScope {
    unsigned long long t0;
    int kind;
    __device__ __forceinline__ explicit TraceScope(int k) : t0(0ull), kind(k) {
        if (threadIdx.x == 0) t0 = global_ns();
    }
    __device__ __forceinline__ ~TraceScope() {
        if (threadIdx.x != 0) return;
        const TraceState ts = g_trace;
        if (ts.rec == nullptr) return;
        const unsigned long long t1 = global_ns();
        unsigned sm;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
        sm %= ts.nsm;
        const unsigned p = atomicAdd(ts.pos + sm, 1u);
        if (p < ts.per_sm)
            ts.rec[(size_t)sm * ts.per_sm + p] = TraceRec{t0, t1, kind, (int)(blockIdx.x + gridDim.x * blockIdx.y),
                                                          (int)sm, (int)(gridDim.x * gridDim.y)};
        else
            atomicAdd(ts.dropped, 1u);
    }
};

}  // namespace fa
