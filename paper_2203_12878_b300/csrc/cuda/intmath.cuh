// Integer semantics of protocol expressions (a reading of the paper's
// unspecified operators, Fig. 1): floor division and Euclidean remainder on
// the 32- or 64-bit arithmetic a protocol was lowered to.  Shared by the
// interpreter and, as text, by the per-protocol kernels compiled at run time.
#pragma once

namespace drf {

// Floor division and Euclidean remainder.  The host's interval analysis
// guarantees b != 0 where no check is made and that no result overflows.
template <typename V, typename U>
__device__ __forceinline__ V floor_div(V a, V b)
{
    V q = a / b;
    V r = (V)((U)a - (U)q * (U)b);
    if (r != 0 && ((r < 0) != (b < 0))) q -= 1;
    return q;
}

template <typename V, typename U>
__device__ __forceinline__ V euclid_mod(V a, V b)
{
    V r = a % b;
    if (r < 0) r = (V)(b > 0 ? (U)r + (U)b : (U)r - (U)b);
    return r;
}

template <typename V> struct Unsigned;
template <> struct Unsigned<int32_t> { using T = uint32_t; };
template <> struct Unsigned<int64_t> { using T = uint64_t; };

}  // namespace drf
