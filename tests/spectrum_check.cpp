// Host-side check of the Chebyshev smoother's spectral estimate
// (csrc/spectrum.cpp): exposes the Hessenberg eigenvalue solver and the
// ellipse fit to tests/test_spectrum.py, which compares them with NumPy's
// eigenvalues and with a fit computed in the test.  Compiled with the
// library's host source only.
#include "common.h"

using namespace hdg;

extern "C" int hess_eigs(const double *H, int n, double *re, double *im) {
    std::vector<double> h(H, H + size_t(n) * n);
    const auto ev = hessenberg_eigenvalues(h, n);
    for (int i = 0; i < n; ++i) {
        re[i] = ev[size_t(i)].real();
        im[i] = ev[size_t(i)].imag();
    }
    return 0;
}

extern "C" int ellipse_fit(const double *re, const double *im, int n, double lower, double grow, double *out) {
    std::vector<std::complex<double>> z;
    for (int i = 0; i < n; ++i) z.emplace_back(re[i], im[i]);
    chebyshev_ellipse(z, lower, grow, out[0], out[1]);
    return 0;
}
