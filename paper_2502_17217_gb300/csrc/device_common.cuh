// Device helpers shared by the library's kernels: deterministic warp/block reductions and the
// last-block grid finalisation (fixed summation order, so every result is bitwise
// reproducible run to run).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace jfnk {

// Programmatic dependent launch (sm_90 and later).  A kernel launched with the
// programmatic-serialisation attribute may start while the kernel before it in the stream is
// still draining; pdl_wait() blocks until that kernel has completed and its memory is
// visible, so every kernel calls it before touching anything earlier work wrote.  Launched
// without the attribute, the wait returns at once.  pdl_trigger() lets the next kernel's
// blocks be scheduled as soon as every block of this grid has issued it.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
#define JF_PDL_ENTRY() \
    do {                 \
        jfnk::pdl_wait();    \
        jfnk::pdl_trigger(); \
    } while (0)

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block; the result is valid in thread 0.  `sh` holds >= blockDim.x/32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = (lane < nw) ? sh[lane] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

// After every block stored partials[b + k * gridDim.x] (k < nvals), the last block to arrive
// returns true; it must then reduce the partials (read with __ldcg) and reset *ticket.
__device__ __forceinline__ bool last_block(unsigned* ticket)
{
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = atomicAdd(ticket, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    return is_last;
}

// Deterministic sum of partials[0..n) by one block (fixed order); result in thread 0.
__device__ __forceinline__ double reduce_partials(const double* partials, int n, double* sh)
{
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += __ldcg(partials + i);
    return block_sum(s, sh);
}

// Of the `expected` blocks that arrive at `ticket` (each after storing its partials), the
// last returns true; it then reads the partials with __ldcg and resets the ticket.
__device__ __forceinline__ bool ticket_last(unsigned* ticket, unsigned expected)
{
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(ticket, 1u) == expected - 1);
    __syncthreads();
    return is_last;
}

// Sum of p[0..count) over one warp in a fixed order, four loads in flight per lane (the
// final sums of a reduction sit on the critical path of every Krylov iteration, so they are
// issued together rather than one dependent L2 round trip at a time); valid in lane 0.
__device__ __forceinline__ double warp_sum_strided(const double* p, int count)
{
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int b0 = 0; b0 < count; b0 += 128) {
        double t[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int b = b0 + 32 * k + lane;
            t[k] = b < count ? __ldcg(p + b) : 0.0;
        }
        s += (t[0] + t[1]) + (t[2] + t[3]);
    }
    return warp_sum(s);
}

// float -> double without the FP64 pipe (on GB300 a conversion costs as much as a DFMA):
// the exponent is re-biased and the mantissa shifted with integer operations.  Exact for
// normal floats and zero; float subnormals (|x| < 1.2e-38) become zero; Inf/NaN become NaN.
__device__ __forceinline__ double f2d(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned a = u & 0x7fffffffu;
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    unsigned long long bits = sign | (((unsigned long long)a << 29) + (896ull << 52));
    bits = (a < 0x00800000u) ? sign : bits;                       // zero and subnormals
    bits = (a >= 0x7f800000u) ? 0x7ff8000000000000ull : bits;     // Inf, NaN
    return __longlong_as_double((long long)bits);
}
__device__ __forceinline__ double to_f64(float f) { return f2d(f); }
__device__ __forceinline__ double to_f64(double d) { return d; }

}  // namespace jfnk
