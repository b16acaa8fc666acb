// Host-side spectral estimate for the Chebyshev smoother: eigenvalues of the
// small upper Hessenberg matrix that a few Arnoldi steps on D^-1 S produce
// (the Ritz values), and the ellipse the Chebyshev iteration is tuned to.
//
// Eigenvalues: the shifted QR algorithm on the Hessenberg matrix in complex
// arithmetic (Givens rotations, Wilkinson shift from the trailing 2 x 2
// block, deflation when a subdiagonal entry falls below machine precision
// relative to its neighbours; an exceptional shift after 10 stalled sweeps).
//
// Ellipse (the reading of the paper's Chebyshev smoother used here): real
// extent [lower b, b] with b = grow * max Re(ritz) (PETSc's default Chebyshev
// bounds are 0.1 and 1.1 times the largest estimate), centre
// theta = (lower b + b) / 2, half-width A; the imaginary semi-axis B is the
// smallest that holds every Ritz value with Re >= lower b, times grow; the
// Chebyshev recurrence needs only theta and delta^2 = A^2 - B^2 (the squared
// focal half-distance, negative for an ellipse taller than wide).
#include "common.h"

#include <cmath>
#include <complex>

namespace hdg {

using cplx = std::complex<double>;

std::vector<cplx> hessenberg_eigenvalues(const std::vector<double> &Hrow, int n) {
    std::vector<cplx> A(size_t(n) * n);
    for (int i = 0; i < n * n; ++i) A[size_t(i)] = Hrow[size_t(i)];
    auto at = [&](int i, int j) -> cplx & { return A[size_t(i) * n + j]; };
    std::vector<cplx> ev(static_cast<size_t>(n));
    const double eps = 2.220446049250313e-16;
    int hi = n - 1, stall = 0;
    while (hi >= 0) {
        if (hi == 0) {
            ev[0] = at(0, 0);
            break;
        }
        // find the active block [lo, hi]
        int lo = hi;
        while (lo > 0) {
            const double s = std::abs(at(lo - 1, lo - 1)) + std::abs(at(lo, lo));
            if (std::abs(at(lo, lo - 1)) <= eps * (s > 0 ? s : 1.0)) {
                at(lo, lo - 1) = 0.0;
                break;
            }
            --lo;
        }
        if (lo == hi) {
            ev[size_t(hi)] = at(hi, hi);
            --hi;
            stall = 0;
            continue;
        }
        // Wilkinson shift: the eigenvalue of the trailing 2 x 2 block closer to its last entry
        const cplx a = at(hi - 1, hi - 1), b = at(hi - 1, hi), c = at(hi, hi - 1), d = at(hi, hi);
        const cplx tr = a + d, det = a * d - b * c;
        const cplx disc = std::sqrt(tr * tr - 4.0 * det);
        const cplx l1 = 0.5 * (tr + disc), l2 = 0.5 * (tr - disc);
        cplx mu = std::abs(l1 - d) < std::abs(l2 - d) ? l1 : l2;
        if (++stall % 11 == 10) mu = d + cplx(0.75 * std::abs(at(hi, hi - 1)), 0.25 * std::abs(at(hi, hi - 1)));
        if (stall > 1000 * n) {          // no convergence: return the diagonal as it stands
            for (int i = 0; i <= hi; ++i) ev[size_t(i)] = at(i, i);
            break;
        }
        // one QR step on the block: H - mu I = Q R, H <- R Q + mu I (Givens)
        std::vector<cplx> cs(static_cast<size_t>(n)), sn(static_cast<size_t>(n));
        for (int i = lo; i <= hi; ++i) at(i, i) -= mu;
        for (int k = lo; k < hi; ++k) {
            const cplx x = at(k, k), y = at(k + 1, k);
            const double r = std::sqrt(std::norm(x) + std::norm(y));
            cplx cc = 1.0, ss = 0.0;
            if (r > 0) {
                cc = x / r;
                ss = y / r;
            }
            cs[size_t(k)] = cc;
            sn[size_t(k)] = ss;
            // rows k, k+1 <- G^H [row k; row k+1]
            for (int j = k; j < n; ++j) {
                const cplx u = at(k, j), v = at(k + 1, j);
                at(k, j) = std::conj(cc) * u + std::conj(ss) * v;
                at(k + 1, j) = -ss * u + cc * v;
            }
        }
        for (int k = lo; k < hi; ++k) {
            const cplx cc = cs[size_t(k)], ss = sn[size_t(k)];
            // columns k, k+1 <- [col k, col k+1] G
            for (int i = 0; i <= std::min(k + 2, hi); ++i) {
                const cplx u = at(i, k), v = at(i, k + 1);
                at(i, k) = u * cc + v * ss;
                at(i, k + 1) = -u * std::conj(ss) + v * std::conj(cc);
            }
        }
        for (int i = lo; i <= hi; ++i) at(i, i) += mu;
    }
    return ev;
}

void chebyshev_ellipse(const std::vector<cplx> &ritz, double lower, double grow, double &theta, double &delta2) {
    double rmax = -1e300;
    for (const cplx &z : ritz) rmax = std::max(rmax, z.real());
    const double b = grow * rmax, a = lower * b;
    const double d = 0.5 * (a + b), A = 0.5 * (b - a);
    double B2 = 0.0;
    for (const cplx &z : ritz) {
        if (z.real() < a) continue;
        const double t = (z.real() - d) / A, q = 1.0 - t * t;
        if (q > 1e-3) B2 = std::max(B2, z.imag() * z.imag() / q);
    }
    B2 *= grow * grow;
    theta = d;
    delta2 = A * A - B2;
}

}  // namespace hdg
