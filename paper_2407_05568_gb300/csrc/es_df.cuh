// es_df.cuh -- double-float arithmetic on the FP32 pipe (a value is hi + lo, two floats: a 48-bit
// significand), and the monitor's density and fundamental derivative evaluated with it.  Used by
// the mixed-precision form's stage, mesh and batched kernels.
//
// The sums and products are the textbook error-free transformations (Knuth's two-sum, Dekker's
// fast two-sum, the FMA residual of a product); the reciprocal is a Newton step on the float one.
#pragma once
#include <cuda_runtime.h>

namespace es {
namespace mixed {

// ---- double-float arithmetic: a value is hi + lo with |lo| <= ulp(hi)/2
struct df {
    float hi, lo;
};
__device__ __forceinline__ df fast_two_sum(float a, float b) {   // |a| >= |b|
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ df df_add(df x, df y) {
    df s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, s.lo + x.lo + y.lo);
}
__device__ __forceinline__ df df_add_f(df x, float y) {
    df s = two_sum(x.hi, y);
    return fast_two_sum(s.hi, s.lo + x.lo);
}
__device__ __forceinline__ df df_mul(df x, df y) {
    const float p = x.hi * y.hi;
    const float e = fmaf(x.hi, y.hi, -p) + (x.hi * y.lo + x.lo * y.hi);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ df df_mul_f(df x, float y) {
    const float p = x.hi * y;
    const float e = fmaf(x.hi, y, -p) + x.lo * y;
    return fast_two_sum(p, e);
}
__device__ __forceinline__ df df_recip(df y) {
    const float q1 = 1.0f / y.hi;
    // r = 1 - q1 y, exactly enough: fma gives the low part of q1 y.hi
    const float r = fmaf(-q1, y.hi, 1.0f) - q1 * y.lo;
    return fast_two_sum(q1, r * q1);
}
__device__ __forceinline__ float df_diff(df a, df b) {            // (a - b) rounded to float
    return (a.hi - b.hi) + (a.lo - b.lo);
}

__device__ __forceinline__ df df_neg(df x) { return {-x.hi, -x.lo}; }

// a double as a (hi, lo) pair of floats
struct df2 {
    float hi, lo;
};
inline df2 split_double(double v) {
    const float hi = float(v);
    return {hi, float(v - double(hi))};
}

// gas constants as (hi, lo) pairs: a, b, 1/c_v, (1 + delta) R and (1 + delta)(2 + delta) R
struct GasDF {
    df2 a, b, icv, k1, k2;
};
inline GasDF gas_df(double a, double b, double R, double cv) {
    const double delta = R / cv;
    GasDF g;
    g.a = split_double(a);
    g.b = split_double(b);
    g.icv = split_double(1.0 / cv);
    g.k1 = split_double((1.0 + delta) * R);
    g.k2 = split_double((1.0 + delta) * (2.0 + delta) * R);
    return g;
}

// Density and fundamental derivative G = nu^3 p_nunu|_s / (2 c^2) (Sec. 1) from a double-float state
// (mass, momenta, energy and J as (hi, lo) pairs), as double-float values.  With nu = 1/rho,
//   G = [(1 + delta)(2 + delta) R T / (1 - b rho)^3 - 6 a rho] / (2 c^2),
//   c^2 = (1 + delta) R T / (1 - b rho)^2 - 2 a rho.
// Near the critical point each bracket is a difference of nearly equal terms (p_nunu: about 16 - 16 =
// -0.02), which FP32 leaves with errors of 1e-5 in G; in double-float both keep ~1e-12.  The monitor
// differentiates both fields, and neighbouring values agree to many digits where the flow is smooth, so
// its differences are formed from these pairs too (df_diff, df_second_diff) before rounding to float.
__device__ __forceinline__ void rho_G_df2(df m0, const df* mom, int dim, df E, df J, const GasDF& G, df* rho_out,
                                          df* G_out) {
    // rho = (J rho) / J; the velocity and the specific energy are quotients of conserved variables, in which J
    // cancels: v = (J rho v) / (J rho), E / rho = (J E) / (J rho)
    const df rho = df_mul(m0, df_recip(J));
    const df im0 = df_recip(m0);
    df ke = {0.0f, 0.0f};
#pragma unroll
    for (int k = 0; k < 3; ++k) {                  // fixed bound: mom[] stays in registers
        if (k < dim) {
            const df v = df_mul(mom[k], im0);
            ke = df_add(ke, df_mul(v, v));
        }
    }
    const df a = {G.a.hi, G.a.lo};
    const df e = df_add(df_mul(E, im0), df_mul_f(df_neg(ke), 0.5f));
    const df T = df_mul(df_add(e, df_mul(rho, a)), {G.icv.hi, G.icv.lo});
    const df om = df_add_f(df_neg(df_mul(rho, {G.b.hi, G.b.lo})), 1.0f);
    const df iom = df_recip(om);
    const df TA = df_mul(T, df_mul(iom, iom));
    const df ar = df_mul(rho, a);
    const df c2 = df_add(df_mul({G.k1.hi, G.k1.lo}, TA), df_mul_f(df_neg(ar), 2.0f));
    const df pnn = df_add(df_mul({G.k2.hi, G.k2.lo}, df_mul(TA, iom)), df_mul_f(df_neg(ar), 6.0f));
    *rho_out = rho;
    *G_out = df_mul(pnn, df_recip(df_mul_f(c2, 2.0f)));
}

// the same, rounded to float
__device__ __forceinline__ void rho_G_df(df m0, const df* mom, int dim, df E, df J, const GasDF& G, float* rho_out,
                                         float* G_out) {
    df r, g;
    rho_G_df2(m0, mom, dim, E, J, G, &r, &g);
    *rho_out = r.hi + r.lo;
    *G_out = g.hi + g.lo;
}

// a_{i+1} - 2 a_i + a_{i-1} of double-float values, rounded to float
__device__ __forceinline__ float df_second_diff(df ap, df a0, df am) {
    return df_diff(df_add(ap, am), df_mul_f(a0, 2.0f));
}

}  // namespace mixed
}  // namespace es
