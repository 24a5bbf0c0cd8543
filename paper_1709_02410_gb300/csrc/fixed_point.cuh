// Deterministic fixed-point accumulation of FP32 matvec contributions.
//
// Every contribution to a blob's velocity (a tile's or a chunk's FP32 sum) is
// scaled by 2^S, rounded to a 64-bit integer and added with an integer atomic
// into one accumulator per blob and component.  Integer addition does not
// depend on its order, so the sum is the same bit for bit whichever order the
// CTAs finish in, with O(n) memory and no reduction kernels.
//
// S is the largest exponent for which no sum can leave 2^61: with cap = the
// largest |velocity component| per unit force and source blob (3 x the
// largest block entry, x 9 with the periodic images), a component is bounded
// by cap n max|F|, and 2^S = 2^61 / (that bound rounded up to a power of two).
// Two's-complement wrap-around makes intermediate overflow harmless as long as
// the final sum fits; the bound leaves a factor of 4 below 2^63.  The rounding
// step 2^-S is at most 2^-60 of the bound.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace rpbd {

// S from the largest finite |force| of the launch; in FP64, where the bound
// stays finite for every finite FP32 force (S then lies within about
// [-130, 210])
__device__ __forceinline__ int fixed_exponent(float fmax, int64_t n, double cap)
{
    const double bound = cap * (double)n * (double)fmax;
    if (!(bound > 0.0)) return 0;
    int e;
    frexp(bound, &e);  // bound < 2^e
    return 61 - e;
}

// adds v 2^S, scaled in two exact FP32 steps 2^h 2^(S-h) so that each factor
// is a normal FP32 number over the whole range of S; a non-finite v
// (non-finite positions) raises flag, and the finishing kernel then writes
// NaN, as a fixed-order reduction of the same sums would
__device__ __forceinline__ void fixed_add(unsigned long long* a, float v, int S, unsigned* flag)
{
    if (!isfinite(v)) {
        atomicExch(flag, 1u);
        return;
    }
    const int h = S >> 1;
    const float s1 = __int_as_float((h + 127) << 23), s2 = __int_as_float((S - h + 127) << 23);
    atomicAdd(a, (unsigned long long)__float2ll_rn((v * s1) * s2));
}

// Folds one thread's largest |force| into fmax_bits[0] (non-negative floats
// order like their bits) and a non-finite force (fm = +inf) into
// fmax_bits[1]; one atomic per warp.  Called by every thread of the warp
// that has not returned.
__device__ __forceinline__ void fixed_force_max(unsigned* fmax_bits, float fm)
{
    const bool bad = isinf(fm);
    const unsigned mask = __activemask();
    const unsigned b = __reduce_max_sync(mask, bad ? 0u : __float_as_uint(fm));
    const unsigned anybad = __any_sync(mask, bad);
    if ((threadIdx.x & 31) == __ffs(mask) - 1) {
        atomicMax(fmax_bits, b);
        if (anybad) atomicExch(fmax_bits + 1, 1u);
    }
}

// U of one system from its accumulators ([3k][n_pad], then the two words of
// fmax_bits): undo 2^S, scale by s_i * inv8pieta and write; NaN everywhere
// when a contribution or a force was not finite.  One thread per (blob,
// component blockIdx.y).
template <class Out>
__global__ void finish_fixed_kernel(int64_t n, int64_t n_pad, int k, double cap,
                                    const unsigned long long* __restrict__ acc, const unsigned* __restrict__ fmax_bits,
                                    const double* __restrict__ scale, double inv8pieta, Out* __restrict__ U)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int q = blockIdx.y;
    if (i >= n || q >= 3 * k) return;
    const int S = fixed_exponent(__uint_as_float(fmax_bits[0]), n, cap);
    const double v = fmax_bits[1] ? __longlong_as_double(0x7ff8000000000000LL)
                                  : ldexp((double)(long long)acc[(int64_t)q * n_pad + i], -S);
    U[(int64_t)q * n + i] = (Out)(scale[i] * inv8pieta * v);
}

}  // namespace rpbd
