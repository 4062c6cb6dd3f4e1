// es_bits.cuh -- float <-> double moves done on the integer and FP32 pipes.
//
// On this GPU the conversion instructions between float and double issue on the FP64 pipe, at 1/64 of the
// FP32 rate, which makes them the bound of the mixed form's elementwise kernels that read or write a double
// per node.  These helpers take the IEEE 754 binary32 / binary64 bit layouts apart with integer operations
// instead (sign, biased exponent, significand; biases 127 and 1023).
#pragma once
#include <cuda_runtime.h>

namespace es {
namespace bits {

// x as an unevaluated sum hi + lo of two floats of x's sign: hi keeps the leading 24 bits of the significand
// (truncated), lo the next 23 of the remaining 29 (truncated), so |x - (hi + lo)| < 2^-46 |x|.  Magnitudes
// outside [2^-103, 2^127) (exponent field outside [920, 1150]), zeros, subnormals, infinities and NaNs take
// the conversion instructions instead.
__device__ __forceinline__ void split(double x, float& hi, float& lo) {
    // the two 32-bit words of x (register moves): sign, 11 exponent bits and significand bits 51..32; bits 31..0
    const unsigned int w1 = (unsigned int)__double2hiint(x), w0 = (unsigned int)__double2loint(x);
    const unsigned int E = (w1 >> 20) & 0x7ffu;
    if (E < 920u || E > 1150u) {
        hi = __double2float_rz(x);
        lo = float(x - double(hi));
        return;
    }
    const unsigned int s = w1 & 0x80000000u;
    const unsigned int m_hi = ((w1 & 0xfffffu) << 3) | (w0 >> 29);      // significand bits 51..29
    const unsigned int m_lo = (w0 & 0x1fffffffu) >> 6;                  // bits 28..6
    hi = __uint_as_float(s | ((E - 896u) << 23) | m_hi);
    // bits 28..6 as the fraction of a float 2^(E-1046) (1 + m_lo 2^-23), less its leading 2^(E-1046): exact
    const float one = __uint_as_float((E - 919u) << 23);
    lo = __uint_as_float(__float_as_uint(__uint_as_float(((E - 919u) << 23) | m_lo) - one) | s);
}

// the double with the value of f (exact for every float: subnormals are normalised, zeros, infinities and
// NaNs keep their class and payload), assembled as two 32-bit words
__device__ __forceinline__ double widen(float f) {
    const unsigned int v = __float_as_uint(f);
    const unsigned int s = v & 0x80000000u;
    const unsigned int e = (v >> 23) & 0xffu;
    const unsigned int m = v & 0x7fffffu;
    unsigned int w1, w0;
    if (e == 0xffu) {
        w1 = s | 0x7ff00000u | (m >> 3);
        w0 = m << 29;
    } else if (e != 0u) {
        w1 = s | ((e + 896u) << 20) | (m >> 3);
        w0 = m << 29;
    } else if (m == 0u) {
        w1 = s;
        w0 = 0u;
    } else {                                // subnormal: m 2^-149 with its leading bit at position p
        const int p = 31 - __clz(m);
        const unsigned int f52 = m << (23 - p);          // the leading bit at position 23, the fraction below it
        w1 = s | ((unsigned int)(p + 874) << 20) | ((f52 & 0x7fffffu) >> 3);
        w0 = f52 << 29;
    }
    return __hiloint2double((int)w1, (int)w0);
}

// the float i for 0 <= i < 2^23 (exact): 2^23 + i from its bits, less 2^23
__device__ __forceinline__ float small_int(int i) {
    return __uint_as_float(0x4b000000u | (unsigned int)i) - 8388608.0f;
}

}  // namespace bits
}  // namespace es
