// FP64 -> FP32 narrowing with integer instructions, for the solvers' FP32 copies of p.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace csrk {
namespace dev {

// GB300 runs the FP32<->FP64 conversion instructions at about the FP64 FMA rate (one warp
// instruction per ~16-20 clocks per SM), so the hot paths convert with integer
// instructions instead.

// FP64 -> FP32 bits, IEEE 754 round to nearest, ties to even, from the bit fields: keep
// the top 23 fraction bits (or, for a subnormal FP32 result, the significand with its
// leading one shifted down to the 2^-149 unit), round on the dropped bits; a carry out of
// the fraction steps the exponent, up to infinity.  FP64 subnormals give a signed zero;
// NaNs stay quiet NaNs.  Agrees bit for bit with the conversion instruction and with the
// host's IEEE conversion on every non-NaN input the tests draw (random patterns over all
// exponents, exact and near ties, subnormal results, range edges: csrk_selftest_narrow).
__device__ __forceinline__ uint32_t f64_to_f32_bits(double d) {
    const uint64_t b = (uint64_t)__double_as_longlong(d);
    const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7FF);
    const uint64_t m = b & 0xFFFFFFFFFFFFFull;
    if (e == 0x7FF) return sign | 0x7F800000u | (m ? 0x400000u | (uint32_t)(m >> 29) : 0u);
    const int ef = e - 1023 + 127;   // FP32 biased exponent
    if (ef >= 255) return sign | 0x7F800000u;
    uint64_t sig;
    int shift;
    uint32_t base;
    if (ef >= 1) {
        sig = m;
        shift = 29;
        base = sign | ((uint32_t)ef << 23);
    } else {
        if (e == 0) return sign;
        shift = 30 - ef;   // value = (2^52 + m) * 2^(e - 1075) = sig * 2^-149 / 2^shift
        if (shift > 63) return sign;
        sig = m | (1ull << 52);
        base = sign;
    }
    const uint64_t kept = sig >> shift;
    const uint64_t rem = sig & ((1ull << shift) - 1);
    const uint64_t half = 1ull << (shift - 1);
    uint32_t r = base + (uint32_t)kept;
    if (rem > half || (rem == half && (kept & 1))) r += 1;
    return r;
}
__device__ __forceinline__ float f64_to_f32(double d) { return __uint_as_float(f64_to_f32_bits(d)); }

}  // namespace dev
}  // namespace csrk
