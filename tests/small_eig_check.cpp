// Reads m, Hs (m x m), Ss (m x m) from stdin, runs the eigensolver's Rayleigh-Ritz step and
// prints the Ritz values and the coefficient matrix (m x r) so the test can check them.
#include <cstdio>
#include <vector>

#include "small_eig.hpp"

int main() {
    int m = 0;
    if (std::scanf("%d", &m) != 1 || m < 1) return 2;
    std::vector<double> Hs(static_cast<size_t>(m) * m), Ss(static_cast<size_t>(m) * m);
    for (double& v : Hs)
        if (std::scanf("%lf", &v) != 1) return 2;
    for (double& v : Ss)
        if (std::scanf("%lf", &v) != 1) return 2;
    std::vector<double> e, Y;
    ndsi::rayleigh_ritz(m, Hs, Ss, e, Y);
    const int r = static_cast<int>(e.size());
    std::printf("%d\n", r);
    for (double v : e) std::printf("%.17g\n", v);
    for (double v : Y) std::printf("%.17g\n", v);
    return 0;
}
