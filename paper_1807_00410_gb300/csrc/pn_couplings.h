// Transport couplings of the real-valued P_N equations, as constexpr closed
// forms read from the paper's appendix ("Final equation": the m = 0, m < 0
// and m > 0 cases; coefficients a..f, beta, delta defined beneath them).
//
// Readings of the printed text (the unreadable or inconsistent spots):
//  * a^{l,m}: the printed denominator (2l+1)(2l-1) gives a^{0,0} = sqrt(-1);
//    the z-recursion coefficient of Y^{l+1,m} has (2l+3)(2l+1), used here.
//  * m > 0, x-derivative of L^{l-1,m-1}: printed with e^{l-1,m-1}; paired
//    with f^{l+1,-m+1} it must be e^{l-1,-m+1} (identical for m = 1).
//  * m > 0, first term: the unknown is L^{l-1,m+1} (dropped in print).
//  * m = 0: two missing "+" signs between terms.
//  * beta^m = sqrt(2) for |m| = 1 else 1; delta_{m != v} as printed.
//  * Terms whose unknown lies outside the truncated expansion are dropped.
// The resulting matrices are those of the Galerkin projection
// int Y_i w_d Y_j in the real SH basis carrying the Condon-Shortley phase.
//
// Everything here is constexpr so that the tiled kernels can bake the
// coefficients into their instruction stream for each order N.
#pragma once

namespace pn {
namespace cpl {

// Square root by Newton's method, usable in constant expressions.
constexpr double csqrt(double v) {
    if (!(v > 0.0)) return 0.0;
    double x = v > 1.0 ? v : 1.0;
    for (int i = 0; i < 200; ++i) {
        const double nx = 0.5 * (x + v / x);
        if (nx == x) break;
        x = nx;
    }
    return x;
}

constexpr double rad(long num, long den) { return num > 0 ? csqrt(double(num) / double(den)) : 0.0; }
constexpr double ca(int l, int m) { return rad(long(l - m + 1) * (l + m + 1), long(2 * l + 3) * (2 * l + 1)); }
constexpr double cb(int l, int m) { return l == 0 ? 0.0 : rad(long(l - m) * (l + m), long(2 * l + 1) * (2 * l - 1)); }
constexpr double cc(int l, int m) { return rad(long(l + m + 1) * (l + m + 2), long(2 * l + 3) * (2 * l + 1)); }
constexpr double cd(int l, int m) { return l == 0 ? 0.0 : rad(long(l - m) * (l - m - 1), long(2 * l + 1) * (2 * l - 1)); }
constexpr double ce(int l, int m) { return rad(long(l - m + 1) * (l - m + 2), long(2 * l + 3) * (2 * l + 1)); }
constexpr double cf(int l, int m) { return l == 0 ? 0.0 : rad(long(l + m) * (l + m - 1), long(2 * l + 1) * (2 * l - 1)); }
constexpr double beta(int m) { return (m == 1 || m == -1) ? 1.4142135623730950488 : 1.0; }

// One transport term of equation (l, m): coef * d/dx_axis L^{lp, mp}.
struct RowTerm {
    int axis;
    int lp, mp;
    double coef;
};

struct RowTerms {
    int n = 0;
    RowTerm t[10] = {};
    constexpr void add(int N, int axis, int lp, int mp, double v) {
        if (lp < 0 || lp > N || mp < -lp || mp > lp) return;
        t[n].axis = axis;
        t[n].lp = lp;
        t[n].mp = mp;
        t[n].coef = v;
        ++n;
    }
};

// The printed terms of equation (l, m) for order N (x = 0, y = 1, z = 2).
constexpr RowTerms row_terms(int N, int l, int m) {
    RowTerms r{};
    const double is2 = 0.70710678118654752440;
    if (m == 0) {
        r.add(N, 0, l - 1, 1, is2 * cc(l - 1, -1));
        r.add(N, 0, l + 1, 1, -is2 * cd(l + 1, -1));
        r.add(N, 1, l - 1, -1, is2 * cc(l - 1, -1));
        r.add(N, 1, l + 1, -1, -is2 * cd(l + 1, -1));
        r.add(N, 2, l - 1, 0, ca(l - 1, 0));
        r.add(N, 2, l + 1, 0, cb(l + 1, 0));
    } else if (m < 0) {
        r.add(N, 1, l - 1, -m + 1, -0.5 * cc(l - 1, m - 1));
        r.add(N, 1, l + 1, -m + 1, 0.5 * cd(l + 1, m - 1));
        r.add(N, 1, l - 1, -m - 1, -0.5 * beta(m) * ce(l - 1, m + 1));
        r.add(N, 1, l + 1, -m - 1, 0.5 * beta(m) * cf(l + 1, m + 1));
        r.add(N, 0, l - 1, m - 1, 0.5 * cc(l - 1, m - 1));
        if (m != -1) {
            r.add(N, 0, l - 1, m + 1, -0.5 * ce(l - 1, m + 1));
            r.add(N, 0, l + 1, m + 1, 0.5 * cf(l + 1, m + 1));
        }
        r.add(N, 0, l + 1, m - 1, -0.5 * cd(l + 1, m - 1));
        r.add(N, 2, l - 1, m, ca(l - 1, m));
        r.add(N, 2, l + 1, m, cb(l + 1, m));
    } else {
        r.add(N, 0, l - 1, m + 1, 0.5 * cc(l - 1, -m - 1));
        r.add(N, 0, l + 1, m + 1, -0.5 * cd(l + 1, -m - 1));
        r.add(N, 0, l - 1, m - 1, -0.5 * beta(m) * ce(l - 1, -m + 1));
        r.add(N, 0, l + 1, m - 1, 0.5 * beta(m) * cf(l + 1, -m + 1));
        r.add(N, 1, l - 1, -m - 1, 0.5 * cc(l - 1, -m - 1));
        r.add(N, 1, l + 1, -m - 1, -0.5 * cd(l + 1, -m - 1));
        if (m != 1) {
            r.add(N, 1, l - 1, -m + 1, 0.5 * ce(l - 1, -m + 1));
            r.add(N, 1, l + 1, -m + 1, -0.5 * cf(l + 1, -m + 1));
        }
        r.add(N, 2, l - 1, m, ca(l - 1, -m));
        r.add(N, 2, l + 1, m, cb(l + 1, -m));
    }
    return r;
}

// Parity bits of coefficient (l, m): the harmonic is odd under reflection of
// axis d exactly when bit d is set; such coefficients sit on cell faces
// along d.
constexpr int parity_class(int l, int m) {
    const int am = m < 0 ? -m : m;
    const int px = m >= 0 ? (m & 1) : ((am + 1) & 1);
    const int py = m < 0 ? 1 : 0;
    const int pz = (l + am) & 1;
    return px + 2 * py + 4 * pz;
}

}  // namespace cpl
}  // namespace pn
