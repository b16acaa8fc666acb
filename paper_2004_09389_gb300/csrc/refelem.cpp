// Reference-element matrices of the library, by Gauss quadrature.
//
// Cell space P^p on the reference triangle (Eq. DG_space_def) with the
// equispaced Lagrange basis written in barycentric product form
//     phi_{ijk} = F_i(L0) F_j(L1) F_k(L2),   F_i(L) = prod_{s<i} (pL - s)/(s+1),
// with (i, j, k) = (p-a-b, a, b) for the node (a/p, b/p).  Trace space P^p on a
// facet (Eq. DG_trace_def) with the 1-D Lagrange basis at t_j = j/p.
// Triangle integrals use the collapsed Gauss-Legendre rule (xi = u,
// eta = v(1-u), weight (1-u)); edge integrals a Gauss-Legendre rule on [0, 1].
// Both are exact for the polynomial degrees involved (<= 2p+1).
#include "common.h"

#include <cmath>

namespace hdg {

namespace {

// Gauss-Legendre nodes and weights on [0, 1] by Newton iteration on P_n.
void gauss_legendre01(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        // recompute derivative at the converged node
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        if (n == 1) { p1 = z; p0 = 1.0; }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = 0.5 * (1.0 - z);
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp);   // 2/((1-z^2)P'^2) on [-1,1], halved
    }
}

// F_i(L) and its derivative dF_i/dL
void factor(int p, int i, double L, double &f, double &df) {
    f = 1.0;
    df = 0.0;
    for (int s = 0; s < i; ++s) {
        double t = (p * L - s) / (s + 1.0);
        double dt = p / (s + 1.0);
        df = df * t + f * dt;
        f *= t;
    }
}

// basis values and xi/eta derivatives at (xi, eta)
void eval_basis(int p, double xi, double eta, std::vector<double> &v, std::vector<double> &dx,
                std::vector<double> &dy) {
    int n = n_cell_nodes(p);
    v.resize(n); dx.resize(n); dy.resize(n);
    double L0 = 1.0 - xi - eta, L1 = xi, L2 = eta;
    int k = 0;
    for (int b = 0; b <= p; ++b) {
        for (int a = 0; a <= p - b; ++a, ++k) {
            int i0 = p - a - b, i1 = a, i2 = b;
            double f0, d0, f1, d1, f2, d2;
            factor(p, i0, L0, f0, d0);
            factor(p, i1, L1, f1, d1);
            factor(p, i2, L2, f2, d2);
            v[k] = f0 * f1 * f2;
            dx[k] = -d0 * f1 * f2 + f0 * d1 * f2;   // dL0/dxi = -1, dL1/dxi = 1
            dy[k] = -d0 * f1 * f2 + f0 * f1 * d2;   // dL0/deta = -1, dL2/deta = 1
        }
    }
}

double trace_basis(int p, int j, double t) {
    double v = 1.0;
    for (int k = 0; k <= p; ++k)
        if (k != j) v *= (t - double(k) / p) / (double(j - k) / p);
    return v;
}

}  // namespace

RefElem build_ref_elem(int p) {
    RefElem r;
    r.p = p;
    r.n = n_cell_nodes(p);
    r.pp = p + 1;
    const int n = r.n, pp = r.pp;
    r.M.assign(n * n, 0.0);
    r.ML.assign(3 * n * n, 0.0);
    r.Dxi.assign(n * n, 0.0);
    r.Deta.assign(n * n, 0.0);
    r.E.assign(3 * n * n, 0.0);
    r.N.assign(3 * n * pp, 0.0);
    r.M1.assign(pp * pp, 0.0);

    std::vector<double> gx, gw;
    gauss_legendre01(p + 3, gx, gw);
    std::vector<double> v, dx, dy;
    for (size_t iu = 0; iu < gx.size(); ++iu) {
        for (size_t iv = 0; iv < gx.size(); ++iv) {
            double xi = gx[iu], eta = gx[iv] * (1.0 - gx[iu]);
            double wt = gw[iu] * gw[iv] * (1.0 - gx[iu]);
            eval_basis(p, xi, eta, v, dx, dy);
            double L[3] = {1.0 - xi - eta, xi, eta};
            for (int a = 0; a < n; ++a) {
                for (int b = 0; b < n; ++b) {
                    double vv = wt * v[a] * v[b];
                    r.M[a * n + b] += vv;
                    for (int i = 0; i < 3; ++i) r.ML[(i * n + a) * n + b] += L[i] * vv;
                    r.Dxi[a * n + b] += wt * v[a] * dx[b];
                    r.Deta[a * n + b] += wt * v[a] * dy[b];
                }
            }
        }
    }
    std::vector<double> ex, ew;
    gauss_legendre01(p + 2, ex, ew);
    const double V[3][2] = {{0.0, 0.0}, {1.0, 0.0}, {0.0, 1.0}};
    for (int i = 0; i < 3; ++i) {
        const double *A = V[(i + 1) % 3], *B = V[(i + 2) % 3];
        for (size_t q = 0; q < ex.size(); ++q) {
            double t = ex[q], wt = ew[q];
            eval_basis(p, A[0] + t * (B[0] - A[0]), A[1] + t * (B[1] - A[1]), v, dx, dy);
            for (int a = 0; a < n; ++a) {
                for (int b = 0; b < n; ++b) r.E[(i * n + a) * n + b] += wt * v[a] * v[b];
                for (int j = 0; j < pp; ++j) r.N[(i * n + a) * pp + j] += wt * v[a] * trace_basis(p, j, t);
            }
        }
    }
    for (size_t q = 0; q < ex.size(); ++q)
        for (int j = 0; j < pp; ++j)
            for (int k = 0; k < pp; ++k)
                r.M1[j * pp + k] += ew[q] * trace_basis(p, j, ex[q]) * trace_basis(p, k, ex[q]);
    return r;
}

std::vector<double> RefElem::packed() const {
    std::vector<double> out;
    out.insert(out.end(), M.begin(), M.end());
    out.insert(out.end(), ML.begin(), ML.end());
    out.insert(out.end(), Dxi.begin(), Dxi.end());
    out.insert(out.end(), Deta.begin(), Deta.end());
    out.insert(out.end(), E.begin(), E.end());
    out.insert(out.end(), N.begin(), N.end());
    out.insert(out.end(), M1.begin(), M1.end());
    return out;
}

}  // namespace hdg
