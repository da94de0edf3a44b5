// Dense transport coupling matrices A_d[k][k'] for the handle's term table,
// from the closed forms in pn_couplings.h (appendix "Final equation").
#include <vector>

#include "pn_couplings.h"
#include "pn_internal.h"

void pn::transport_couplings(int N, std::vector<double>& A) {
    const int K = (N + 1) * (N + 1);
    A.assign(size_t(3) * K * K, 0.0);
    for (int l = 0; l <= N; ++l)
        for (int m = -l; m <= l; ++m) {
            const cpl::RowTerms r = cpl::row_terms(N, l, m);
            const int k = l * l + l + m;
            for (int i = 0; i < r.n; ++i) {
                const int kp = r.t[i].lp * r.t[i].lp + r.t[i].lp + r.t[i].mp;
                A[(size_t(r.t[i].axis) * K + k) * K + kp] += r.t[i].coef;
            }
        }
}
