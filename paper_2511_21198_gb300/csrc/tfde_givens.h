// Givens-rotated least-squares state of one GMRES cycle (host, FP64): the
// small (m+1) x m Hessenberg problem min || beta e_1 - H y || of the Arnoldi
// process (Sec. 3.2), shared by the FP64 and the mixed-precision PGMRES.
#pragma once

#include <cmath>
#include <vector>

namespace tfde {

struct GivensLS {
    int m;
    std::vector<double> R, cs, sn, g;
    explicit GivensLS(int m_) : m(m_), R((size_t)(m_ + 1) * m_, 0.0), cs(m_), sn(m_), g(m_ + 1, 0.0) {}
    double& at(int i, int j) { return R[(size_t)i * m + j]; }
    // column j of the Hessenberg matrix (entries 0..j+1) -> rotated; returns |g_{j+1}|
    double add_column(int j, const double* h) {
        for (int i = 0; i <= j + 1; ++i) at(i, j) = h[i];
        for (int i = 0; i < j; ++i) {
            const double t = cs[i] * at(i, j) + sn[i] * at(i + 1, j);
            at(i + 1, j) = -sn[i] * at(i, j) + cs[i] * at(i + 1, j);
            at(i, j) = t;
        }
        const double den = std::hypot(at(j, j), at(j + 1, j));
        cs[j] = den > 0.0 ? at(j, j) / den : 1.0;
        sn[j] = den > 0.0 ? at(j + 1, j) / den : 0.0;
        at(j, j) = den;
        at(j + 1, j) = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        return std::fabs(g[j + 1]);
    }
    void solve(int k, std::vector<double>& y) {
        y.assign(k, 0.0);
        for (int i = k - 1; i >= 0; --i) {
            double t = g[i];
            for (int j = i + 1; j < k; ++j) t -= at(i, j) * y[j];
            y[i] = t / at(i, i);
        }
    }
};

}  // namespace tfde
