// Transport coupling table of the real-valued P_N equations, read from the
// closed forms of the paper's appendix ("Final equation": the m = 0, m < 0
// and m > 0 cases, with coefficients a..f, beta, delta defined beneath them).
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
// int Y_i w_d Y_j in the real SH basis that carries the Condon-Shortley phase.
#include <cmath>
#include <vector>

#include "pn_internal.h"

namespace {

double rad(double v) { return v > 0.0 ? std::sqrt(v) : 0.0; }

double ca(int l, int m) { return rad(double((l - m + 1) * (l + m + 1)) / double((2 * l + 3) * (2 * l + 1))); }
double cb(int l, int m) { return l == 0 ? 0.0 : rad(double((l - m) * (l + m)) / double((2 * l + 1) * (2 * l - 1))); }
double cc(int l, int m) { return rad(double((l + m + 1) * (l + m + 2)) / double((2 * l + 3) * (2 * l + 1))); }
double cd(int l, int m) { return l == 0 ? 0.0 : rad(double((l - m) * (l - m - 1)) / double((2 * l + 1) * (2 * l - 1))); }
double ce(int l, int m) { return rad(double((l - m + 1) * (l - m + 2)) / double((2 * l + 3) * (2 * l + 1))); }
double cf(int l, int m) { return l == 0 ? 0.0 : rad(double((l + m) * (l + m - 1)) / double((2 * l + 1) * (2 * l - 1))); }
double beta(int m) { return (m == 1 || m == -1) ? std::sqrt(2.0) : 1.0; }

struct Acc {
    int N, K;
    std::vector<double>& A;
    void add(int l, int m, int axis, int lp, int mp, double v) {
        if (lp < 0 || lp > N) return;
        if (mp < -lp || mp > lp) return;
        int k = l * l + l + m, kp = lp * lp + lp + mp;
        A[(size_t(axis) * K + k) * K + kp] += v;
    }
};

}  // namespace

void pn::transport_couplings(int N, std::vector<double>& A) {
    const int K = (N + 1) * (N + 1);
    A.assign(size_t(3) * K * K, 0.0);
    Acc acc{N, K, A};
    const double is2 = 1.0 / std::sqrt(2.0);
    enum { X = 0, Y = 1, Z = 2 };
    for (int l = 0; l <= N; ++l) {
        for (int m = -l; m <= l; ++m) {
            if (m == 0) {
                acc.add(l, m, X, l - 1, 1, is2 * cc(l - 1, -1));
                acc.add(l, m, X, l + 1, 1, -is2 * cd(l + 1, -1));
                acc.add(l, m, Y, l - 1, -1, is2 * cc(l - 1, -1));
                acc.add(l, m, Y, l + 1, -1, -is2 * cd(l + 1, -1));
                acc.add(l, m, Z, l - 1, 0, ca(l - 1, 0));
                acc.add(l, m, Z, l + 1, 0, cb(l + 1, 0));
            } else if (m < 0) {
                acc.add(l, m, Y, l - 1, -m + 1, -0.5 * cc(l - 1, m - 1));
                acc.add(l, m, Y, l + 1, -m + 1, 0.5 * cd(l + 1, m - 1));
                acc.add(l, m, Y, l - 1, -m - 1, -0.5 * beta(m) * ce(l - 1, m + 1));
                acc.add(l, m, Y, l + 1, -m - 1, 0.5 * beta(m) * cf(l + 1, m + 1));
                acc.add(l, m, X, l - 1, m - 1, 0.5 * cc(l - 1, m - 1));
                if (m != -1) {
                    acc.add(l, m, X, l - 1, m + 1, -0.5 * ce(l - 1, m + 1));
                    acc.add(l, m, X, l + 1, m + 1, 0.5 * cf(l + 1, m + 1));
                }
                acc.add(l, m, X, l + 1, m - 1, -0.5 * cd(l + 1, m - 1));
                acc.add(l, m, Z, l - 1, m, ca(l - 1, m));
                acc.add(l, m, Z, l + 1, m, cb(l + 1, m));
            } else {
                acc.add(l, m, X, l - 1, m + 1, 0.5 * cc(l - 1, -m - 1));
                acc.add(l, m, X, l + 1, m + 1, -0.5 * cd(l + 1, -m - 1));
                acc.add(l, m, X, l - 1, m - 1, -0.5 * beta(m) * ce(l - 1, -m + 1));
                acc.add(l, m, X, l + 1, m - 1, 0.5 * beta(m) * cf(l + 1, -m + 1));
                acc.add(l, m, Y, l - 1, -m - 1, 0.5 * cc(l - 1, -m - 1));
                acc.add(l, m, Y, l + 1, -m - 1, -0.5 * cd(l + 1, -m - 1));
                if (m != 1) {
                    acc.add(l, m, Y, l - 1, -m + 1, 0.5 * ce(l - 1, -m + 1));
                    acc.add(l, m, Y, l + 1, -m + 1, -0.5 * cf(l + 1, -m + 1));
                }
                acc.add(l, m, Z, l - 1, m, ca(l - 1, -m));
                acc.add(l, m, Z, l + 1, m, cb(l + 1, -m));
            }
        }
    }
}
