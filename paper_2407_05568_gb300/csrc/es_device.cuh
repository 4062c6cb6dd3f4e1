// es_device.cuh -- device-side physics of the ES van der Waals scheme (sm_103a).
//
// Everything here runs inside the library's own kernels.  Formulas follow the
// paper's sections noted at each function, written in general van der Waals
// units (a, b, R, cv): p = rho R T/(1 - b rho) - a rho^2, e = cv T - a rho.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "es_vdw.h"

namespace es {

// ----------------------------------------------------------------- constants
struct Gas {
    double a, b, R, cv, delta;   // delta = R / cv
    double iR, idelta, icv;      // 1/R, 1/delta, 1/cv (set with the others)
};

inline void gas_reciprocals(Gas& g) {
    g.iR = 1.0 / g.R;
    g.idelta = 1.0 / g.delta;
    g.icv = 1.0 / g.cv;
}

// Reciprocal and quotient for finite, normal, nonzero divisors (all the kernels' divisors are
// positive physical quantities or sums of them): the hardware's approximate reciprocal refined by
// two Newton-Raphson steps, y <- y + y (1 - b y), each of which squares the relative error, and
// for the quotient one correction q <- q + y (a - b q) (Markstein, IBM J. Res. Develop. 34(1),
// 1990).  Checked against IEEE division on the GPU (es_selftest_division).
__device__ __forceinline__ double rcp_nr(double b) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(b));
    y = fma(y, fma(-b, y, 1.0), y);
    y = fma(y, fma(-b, y, 1.0), y);
    return y;
}
__device__ __forceinline__ double div_nr(double a, double b) {
    const double y = rcp_nr(b);
    const double q = a * y;
    return fma(fma(-b, q, a), y, q);
}

// Sixth-order EC combination weights alpha_{3,m}, m = 1, 2, 3 (Sec. 3.1:
// sum m alpha = 1, sum m^3 alpha = sum m^5 alpha = 0).
__device__ __forceinline__ double ec_alpha(int m) {
    return m == 1 ? 1.5 : (m == 2 ? -0.3 : 1.0 / 30.0);
}

// ------------------------------------------------------------ log mean
// Reciprocal of the logarithmic mean {a}^ln = [[a]]/[[ln a]] (Sec. 3.1), from
// per-node logarithms.  When |f| = |a_l - a_r|/(a_l + a_r) < 1e-2 the quotient
// of differences loses digits, so the Taylor series of artanh(f)/f is used:
// 1/{a}^ln = 2 F(f)/(a_l + a_r), F = 1 + f^2/3 + f^4/5 + ... (six terms).
__device__ __forceinline__ double inv_log_mean(double al, double ar, double lnl, double lnr) {
    const double s = al + ar;
    const double d = al - ar;
    if (fabs(d) < 1e-2 * s) {
        const double is = rcp_nr(s);
        const double f = d * is;
        const double u = f * f;
        const double F = 1.0 + u * (1.0 / 3.0 + u * (1.0 / 5.0 + u * (1.0 / 7.0 + u * (1.0 / 9.0 + u * (1.0 / 11.0)))));
        return 2.0 * F * is;
    }
    return div_nr(lnl - lnr, d);
}

// --------------------------------------------------------- MR-WENO5 (Sec. 3.3)
// Multi-resolution WENO on the nested stencils {0}, {-1,0,1}, {-2..2} (Zhu & Shu
// framework) reconstructing the value at x_{i+1/2} from point values treated as
// cell averages.  g1, g2, g3 = linear weights of the 1-, 3-, 5-point stencils.
struct Weno {
    double g1, g2, g3;     // linear weights
    double g12, ig22;      // g1/(g1+g2), (g1+g2)/g2
    double ig3;            // 1/g3
    double eps;
    double sign_tol;       // relative round-off size under which a plain jump counts as zero
};

__device__ __forceinline__ double mr_weno5(double wm2, double wm1, double w0, double wp1, double wp2,
                                           const Weno& c) {
    // candidate interface values
    const double q2 = (-wm1 + 5.0 * w0 + 2.0 * wp1) * (1.0 / 6.0);
    const double q3 = (2.0 * wm2 - 13.0 * wm1 + 47.0 * w0 + 27.0 * wp1 - 3.0 * wp2) * (1.0 / 60.0);
    const double p1 = w0;
    const double p2 = (q2 - c.g12 * p1) * c.ig22;
    const double p3 = (q3 - c.g1 * p1 - c.g2 * p2) * c.ig3;
    // smoothness: beta_1 from the two one-sided differences
    const double dl = w0 - wm1, dr = wp1 - w0;
    const double b1 = fmin(dl * dl, dr * dr);
    // beta_2: sum_alpha int (d^alpha q)^2 of the quadratic on the cell
    const double s2a = wm1 - 2.0 * w0 + wp1, s2b = wp1 - wm1;
    const double b2 = (13.0 / 12.0) * s2a * s2a + 0.25 * s2b * s2b;
    // beta_3: coefficients c1..c4 of the quartic q(x) = sum c_k x^k (unit cell
    // centred at 0) whose cell averages are w_{-2..2}; odd part from
    // o1 = (w1 - w-1)/2, o2 = (w2 - w-2)/2, even part from the means of w_{+-1} and
    // w_{+-2} relative to w0 (beta ignores a constant added to the data, so everything is
    // formed from differences: no rounding of |w|-sized terms in small indicators)
    const double o1 = 0.5 * (wp1 - wm1), o2 = 0.5 * (wp2 - wm2);
    const double a1 = 0.5 * ((wp1 - w0) + (wm1 - w0)), a2 = 0.5 * ((wp2 - w0) + (wm2 - w0));
    const double c3 = (o2 - 2.0 * o1) * (1.0 / 6.0);
    const double c1 = (34.0 * o1 - 5.0 * o2) * (1.0 / 24.0);
    const double c4 = (a2 - 4.0 * a1) * (1.0 / 12.0);
    const double c2 = (12.0 * a1 - a2) * 0.125;
    // int_{-1/2}^{1/2} of (q')^2 + (q'')^2 + (q''')^2 + (q'''')^2 (int x^2 = 1/12, x^4 = 1/80,
    // x^6 = 1/448), collected by monomial: c1^2 + c1 c3/2 + 13/3 c2^2 + 3129/80 c3^2
    // + 21/5 c2 c4 + 87617/140 c4^2
    const double b3 = c1 * (c1 + 0.5 * c3) + c2 * ((13.0 / 3.0) * c2 + 4.2 * c4) + (3129.0 / 80.0) * c3 * c3
                    + (87617.0 / 140.0) * c4 * c4;
    const double t = 0.5 * (fabs(b3 - b1) + fabs(b3 - b2));
    const double tau = t * t;
    // w~_l = g_l (1 + tau/(beta_l + eps)); scaled by (d1 d2 d3) to need one division
    const double d1 = b1 + c.eps, d2 = b2 + c.eps, d3 = b3 + c.eps;
    const double n1 = c.g1 * (d1 + tau) * (d2 * d3);
    const double n2 = c.g2 * (d2 + tau) * (d1 * d3);
    const double n3 = c.g3 * (d3 + tau) * (d1 * d2);
    return div_nr(n1 * p1 + n2 * p2 + n3 * p3, n1 + n2 + n3);
}

// --------------------------------------------------------- index helpers
__device__ __forceinline__ int wrap_index(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

// Decomposition of a possibly-ghost index along one direction into at most two
// interior indices with weights and a period count:
//   periodic: value(i) = value(i mod n) + q * period
//   outflow : value(i) = 2 value(boundary) - value(mirror)   (odd reflection)
struct GhostTerms {
    int idx[2];
    double w[2];
    int nterm;
    int q;         // period count (periodic only)
};

// Walls and symmetry planes: the end of a direction that mirrors the mesh and the state.
__device__ __forceinline__ bool end_mirrored(int bc, bool lo) {
    return bc == ES_BC_REFLECT || (bc == ES_BC_SYMMETRY_LO && lo);
}

// `tangential`: a coordinate or mesh-velocity component along the boundary plane, which a
// mirroring end mirrors (value of the mirror node) instead of reflecting oddly.
__device__ __forceinline__ GhostTerms ghost_terms(int i, int n, int bc, bool tangential = false) {
    GhostTerms g;
    g.q = 0;
    if (i >= 0 && i < n) {
        g.idx[0] = i; g.w[0] = 1.0; g.nterm = 1;
    } else if (bc == ES_BC_PERIODIC) {
        int r = wrap_index(i, n);
        g.q = (i - r) / n;
        g.idx[0] = r; g.w[0] = 1.0; g.nterm = 1;
    } else {
        // the mirror index is clamped to the mesh: nodes that far out only
        // occur in the unused tail of a ragged tile and must stay in bounds
        int m = i < 0 ? -i : 2 * (n - 1) - i;
        m = m < 0 ? 0 : (m > n - 1 ? n - 1 : m);
        if (tangential && end_mirrored(bc, i < 0)) {
            g.idx[0] = m; g.w[0] = 1.0; g.nterm = 1;
        } else {
            g.idx[0] = i < 0 ? 0 : n - 1; g.w[0] = 2.0; g.idx[1] = m; g.w[1] = -1.0; g.nterm = 2;
        }
    }
    return g;
}

// State index for ghosts: periodic wrap, outflow copy of the boundary node, mirror node at a
// wall or symmetry end (the caller negates the normal momentum there).
__device__ __forceinline__ int state_index(int i, int n, int bc) {
    if (i >= 0 && i < n) return i;
    if (bc == ES_BC_PERIODIC) return wrap_index(i, n);
    if (end_mirrored(bc, i < 0)) {
        int m = i < 0 ? -i : 2 * (n - 1) - i;
        return m < 0 ? 0 : (m > n - 1 ? n - 1 : m);
    }
    return i < 0 ? 0 : n - 1;
}

// ------------------------------------------------------------- reductions
// Atomic max / min of non-negative doubles through their ordered bit patterns.
__device__ __forceinline__ void atomic_max_pos(unsigned long long* addr, double v) {
    if (!(v >= 0.0)) v = __longlong_as_double(0x7ff0000000000000ULL);   // NaN -> +inf
    atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ void atomic_min_pos(unsigned long long* addr, double v) {
    if (!(v >= 0.0)) v = 0.0;
    atomicMin(addr, (unsigned long long)__double_as_longlong(v));
}

// Device error word: first error code wins; the node index is kept with it.
struct DevStatus {
    int code;
    int index;
};

__device__ __forceinline__ void raise_error(DevStatus* st, int code, int index) {
    if (atomicCAS(&st->code, 0, code) == 0) st->index = index;
}

}  // namespace es
