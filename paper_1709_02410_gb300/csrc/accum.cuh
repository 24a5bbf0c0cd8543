// Compensated FP32 summation for the reductions of FP32 tile partials.
//
// A running sum is kept as an unevaluated pair s + c of floats: each
// addition's rounding error is recovered exactly by Knuth's two-sum and
// collected in c.  The pair carries about 48 significant bits, like an FP64
// accumulator, but every operation runs on the FP32 pipe (FP64 throughput on
// this GPU is a small fraction of FP32).  The pair is widened to FP64 once,
// at the end of the sum.
#pragma once

#include <cuda_runtime.h>

namespace rpbd {

// s + c += x; the _rn intrinsics keep the compiler from contracting or
// reassociating the error terms
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float x)
{
    const float t = __fadd_rn(s, x);
    const float bp = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
    s = t;
    c = __fadd_rn(c, e);
}

__device__ __forceinline__ double two_sum_value(float s, float c) { return (double)s + (double)c; }

}  // namespace rpbd
