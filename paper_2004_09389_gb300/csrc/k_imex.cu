// IMEX time stepping around the implicit solve (Sec. 3.3, Eqs. theta_method,
// IMEX_HDG_I and IMEX_HDG_II; tableaux of Sec. 5.1).
//
// The semi-discrete system is M dq/dt = N(q) + L(q): L holds the gravity-wave
// terms with the upwind stabilisation (taken implicitly), N the Coriolis term
// (taken explicitly, as in the paper).  Everything here works on nodal
// function values (the caller's u [N][2][n_p], h [N][n_p] layout), so each
// mass matrix is applied through its inverse per cell:
//   n~(q) = M^-1 N(q),  l~(q) = M^-1 L(q).
// An implicit stage M Q - a~_ii dt L(Q) = M r is the hot path's solve with
// f = 0 and tau = a~_ii dt, right-hand-side function r (hdg_solve_dev +
// hdg_recover_dev).  L is evaluated from the DG state: the trace on each facet
// is the upwind value lambda = {h} + H / (2 tau_s) (u_1.n_1 + u_2.n_2) (the
// HDG transmission condition solved pointwise; every trace is in P^p(e)), and
// per cell, in the integrated-by-parts form of the library's condensation,
//   L_u(q) . w  = g (h, div w) - g <lambda, w.n>_dK
//   L_h(q) psi  = -H (div u, psi) - tau_s <h - lambda, psi>_dK
//   N_u(q) . w  = -(f u_perp, w),  N_h = 0,   u_perp = (-u_y, u_x).
#include "common.h"

#include <algorithm>
#include <cmath>

namespace hdg {
namespace {

inline unsigned nblocks(size_t n, int bs) { return unsigned((n + bs - 1) / bs); }

// index of the cell node at edge i, position j (edge from local vertex
// (i+1)%3 to (i+2)%3); nodes (a/p, b/p) are numbered b outer, a inner
template <int P>
__device__ __forceinline__ int edge_node(int i, int j) {
    int a, b;
    if (i == 0) { a = P - j; b = j; }
    else if (i == 1) { a = 0; b = P - j; }
    else { a = j; b = 0; }
    return b * (P + 1) - b * (b - 1) / 2 + a;
}

// outward unit normal of edge i of a counter-clockwise cell with local vertices x[6]
__device__ __forceinline__ void edge_normal(const double *x, int i, double &nx, double &ny, double &len) {
    const int v1 = (i + 1) % 3, v2 = (i + 2) % 3;
    const double tx = x[2 * v2] - x[2 * v1], ty = x[2 * v2 + 1] - x[2 * v1 + 1];
    len = sqrt(tx * tx + ty * ty);
    nx = ty / len;
    ny = -tx / len;
}

// lambda at the p+1 trace nodes of every facet (internal layout [PP][NF])
template <int P>
__global__ void upwind_trace_kernel(int NF, const int32_t *__restrict__ fcell, const int32_t *__restrict__ fedge,
                                    const int32_t *__restrict__ flip, const double *__restrict__ X,
                                    const double *__restrict__ u, const double *__restrict__ h, double H, double ts,
                                    double *__restrict__ lam) {
    constexpr int PP = P + 1, NP = (P + 1) * (P + 2) / 2;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NF) return;
    double v[PP];
#pragma unroll
    for (int r = 0; r < PP; ++r) v[r] = 0.0;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int K = fcell[2 * e + s], i = fedge[2 * e + s], fl = flip[3 * K + i];
        double x[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) x[k] = X[size_t(K) * 6 + k];
        double nx, ny, len;
        edge_normal(x, i, nx, ny, len);
#pragma unroll
        for (int r = 0; r < PP; ++r) {
            const int node = edge_node<P>(i, fl ? P - r : r);
            const double hv = h[size_t(K) * NP + node];
            const double un = nx * u[size_t(K) * 2 * NP + node] + ny * u[size_t(K) * 2 * NP + NP + node];
            v[r] += 0.5 * hv + (H / (2.0 * ts)) * un;
        }
    }
#pragma unroll
    for (int r = 0; r < PP; ++r) lam[size_t(r) * NF + e] = v[r];
}

struct RateArgs {
    int N, NF;
    double g, H, ts;
    const double *ref;       // packed reference matrices
    const double *minv;      // [NP][NP] inverse of the reference mass matrix
    const double *X;         // [N][3][2]
    const double *fcell;     // [N][3] Coriolis at the cell's vertices (P1), or null
    const int32_t *facet_of, *flip;
    const double *lam;       // [PP][NF]
    const double *u, *h;     // state
    double *nu, *nh;         // M^-1 N(q) (u and h parts), or null
    double *lu, *lh;         // M^-1 L(q)
};

// one thread per cell: the cell's rows of L(q) and N(q), then the inverse
// cell mass matrix (M_K = |det J| M_ref)
template <int P>
__global__ void __launch_bounds__(128) imex_rates_kernel(RateArgs a) {
    constexpr int PP = P + 1, NP = (P + 1) * (P + 2) / 2;
    constexpr int oM = 0, oML = oM + NP * NP, oDxi = oML + 3 * NP * NP, oDeta = oDxi + NP * NP,
                  oE = oDeta + NP * NP, oN = oE + 3 * NP * NP, oM1 = oN + 3 * NP * PP, oEnd = oM1 + PP * PP;
    __shared__ double ref[oEnd];
    __shared__ double minv[NP * NP];
    for (int k = threadIdx.x; k < oEnd; k += blockDim.x) ref[k] = a.ref[k];
    for (int k = threadIdx.x; k < NP * NP; k += blockDim.x) minv[k] = a.minv[k];
    __syncthreads();
    const int K = blockIdx.x * blockDim.x + threadIdx.x;
    if (K >= a.N) return;
    double x[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) x[k] = a.X[size_t(K) * 6 + k];
    const double J00 = x[2] - x[0], J01 = x[4] - x[0], J10 = x[3] - x[1], J11 = x[5] - x[1];
    const double det = J00 * J11 - J01 * J10;
    // J^-T: d/dx = j00 d/dxi + j01 d/deta, d/dy = j10 d/dxi + j11 d/deta
    const double j00 = J11 / det, j01 = -J10 / det, j10 = -J01 / det, j11 = J00 / det;
    double ux[NP], uy[NP], hh[NP];
#pragma unroll
    for (int b = 0; b < NP; ++b) {
        ux[b] = a.u[size_t(K) * 2 * NP + b];
        uy[b] = a.u[size_t(K) * 2 * NP + NP + b];
        hh[b] = a.h[size_t(K) * NP + b];
    }
    double lam[3][PP], nrm[3][2], len[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        edge_normal(x, i, nrm[i][0], nrm[i][1], len[i]);
        const int f = a.facet_of[3 * K + i], fl = a.flip[3 * K + i];
#pragma unroll
        for (int j = 0; j < PP; ++j) lam[i][j] = a.lam[size_t(fl ? P - j : j) * a.NF + f];
    }
    const double g = a.g, H = a.H, ts = a.ts;
    // L(q) rows, tested against phi_a
    double Lx[NP], Ly[NP], Lh[NP];
#pragma unroll
    for (int ia = 0; ia < NP; ++ia) {
        double lx = 0.0, ly = 0.0, lh = 0.0;
#pragma unroll
        for (int ib = 0; ib < NP; ++ib) {
            // g (h, d_x phi_a) = g sum_b h_b int phi_b d_x phi_a
            const double dxi_ba = ref[oDxi + ib * NP + ia], deta_ba = ref[oDeta + ib * NP + ia];
            lx = fma(g * det * (j00 * dxi_ba + j01 * deta_ba), hh[ib], lx);
            ly = fma(g * det * (j10 * dxi_ba + j11 * deta_ba), hh[ib], ly);
            // -H (div u, phi_a) = -H sum_b (u_x,b int phi_a d_x phi_b + u_y,b int phi_a d_y phi_b)
            const double dxi_ab = ref[oDxi + ia * NP + ib], deta_ab = ref[oDeta + ia * NP + ib];
            lh = fma(-H * det * (j00 * dxi_ab + j01 * deta_ab), ux[ib], lh);
            lh = fma(-H * det * (j10 * dxi_ab + j11 * deta_ab), uy[ib], lh);
            // -tau_s <h, phi_a>_dK
            double e = 0.0;
#pragma unroll
            for (int i = 0; i < 3; ++i) e = fma(len[i], ref[oE + (i * NP + ia) * NP + ib], e);
            lh = fma(-ts * e, hh[ib], lh);
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            double nl = 0.0;
#pragma unroll
            for (int j = 0; j < PP; ++j) nl = fma(ref[oN + (i * NP + ia) * PP + j], lam[i][j], nl);
            nl *= len[i];
            lx = fma(-g * nrm[i][0], nl, lx);      // -g <lambda, w.n>
            ly = fma(-g * nrm[i][1], nl, ly);
            lh = fma(ts, nl, lh);                  // + tau_s <lambda, psi>
        }
        Lx[ia] = lx;
        Ly[ia] = ly;
        Lh[ia] = lh;
    }
    // M_K^-1 = M_ref^-1 / det
    const double s = 1.0 / det;
#pragma unroll
    for (int ia = 0; ia < NP; ++ia) {
        double vx = 0.0, vy = 0.0, vh = 0.0;
#pragma unroll
        for (int ib = 0; ib < NP; ++ib) {
            const double mi = minv[ia * NP + ib];
            vx = fma(mi, Lx[ib], vx);
            vy = fma(mi, Ly[ib], vy);
            vh = fma(mi, Lh[ib], vh);
        }
        a.lu[size_t(K) * 2 * NP + ia] = s * vx;
        a.lu[size_t(K) * 2 * NP + NP + ia] = s * vy;
        a.lh[size_t(K) * NP + ia] = s * vh;
    }
    if (!a.nu) return;
    // N(q) = -(f u_perp, w): x row +(f u_y, phi_a), y row -(f u_x, phi_a); f is P1
    double f0 = a.fcell[size_t(K) * 3], f1 = a.fcell[size_t(K) * 3 + 1], f2 = a.fcell[size_t(K) * 3 + 2];
#pragma unroll
    for (int ia = 0; ia < NP; ++ia) {
        double nx = 0.0, ny = 0.0;
#pragma unroll
        for (int ib = 0; ib < NP; ++ib) {
            const double mf = det * (f0 * ref[oML + ia * NP + ib] + f1 * ref[oML + NP * NP + ia * NP + ib] +
                                     f2 * ref[oML + 2 * NP * NP + ia * NP + ib]);
            nx = fma(mf, uy[ib], nx);
            ny = fma(-mf, ux[ib], ny);
        }
        Lx[ia] = nx;
        Ly[ia] = ny;
    }
#pragma unroll
    for (int ia = 0; ia < NP; ++ia) {
        double vx = 0.0, vy = 0.0;
#pragma unroll
        for (int ib = 0; ib < NP; ++ib) {
            const double mi = minv[ia * NP + ib];
            vx = fma(mi, Lx[ib], vx);
            vy = fma(mi, Ly[ib], vy);
        }
        a.nu[size_t(K) * 2 * NP + ia] = s * vx;
        a.nu[size_t(K) * 2 * NP + NP + ia] = s * vy;
        a.nh[size_t(K) * NP + ia] = 0.0;
    }
}

// out = q0 + dt sum_j (cn[j] n~_j + cl[j] l~_j), over whole state vectors
// (u part then h part, n entries); coefficients that are 0 are skipped
struct Combo {
    int k;
    double cn[8], cl[8];
    const double *n[8], *l[8];
};
__global__ void imex_combine_kernel(size_t n, const double *__restrict__ q0, Combo c, double dt,
                                    double *__restrict__ out) {
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = 0.0;
    for (int j = 0; j < c.k; ++j) {
        if (c.cn[j] != 0.0) acc = fma(c.cn[j], c.n[j][i], acc);
        if (c.cl[j] != 0.0) acc = fma(c.cl[j], c.l[j][i], acc);
    }
    out[i] = fma(dt, acc, q0[i]);
}

// Butcher tableaux (explicit a, implicit a~, weights b, b~) of Sec. 5.1
struct Tableau {
    int s;
    double a[5][5], at[5][5], b[5], bt[5];
};

Tableau tableau(int scheme, double theta) {
    Tableau T{};
    if (scheme == HDG_IMEX_THETA) {
        // M q1 = M q0 + dt (N(q0) + (1 - theta) L(q0) + theta L(q1)) as a
        // two-stage method: Q_1 = q0 (explicit), Q_2 implicit with a~_22 = theta
        T.s = 2;
        T.a[1][0] = 1.0;
        T.at[1][0] = 1.0 - theta;
        T.at[1][1] = theta;
        T.b[0] = 1.0;
        T.bt[0] = 1.0 - theta;
        T.bt[1] = theta;
    } else if (scheme == HDG_IMEX_ARS2) {
        const double g = 1.0 - 1.0 / std::sqrt(2.0), d = -2.0 * std::sqrt(2.0) / 3.0;
        T.s = 3;
        T.a[1][0] = g;
        T.a[2][0] = d; T.a[2][1] = 1.0 - d;
        T.at[1][1] = g;
        T.at[2][1] = 1.0 - g; T.at[2][2] = g;
        T.b[1] = 1.0 - g; T.b[2] = g;
        T.bt[1] = 1.0 - g; T.bt[2] = g;
    } else if (scheme == HDG_IMEX_SSP2) {
        T.s = 3;
        T.a[2][1] = 1.0;
        T.at[0][0] = 0.5;
        T.at[1][0] = -0.5; T.at[1][1] = 0.5;
        T.at[2][1] = 0.5; T.at[2][2] = 0.5;
        T.b[1] = 0.5; T.b[2] = 0.5;
        T.bt[1] = 0.5; T.bt[2] = 0.5;
    } else {   // ARS3(4,4,3)
        T.s = 5;
        const double A[5][5] = {{0, 0, 0, 0, 0}, {0.5, 0, 0, 0, 0}, {11.0 / 18, 1.0 / 18, 0, 0, 0},
                                {5.0 / 6, -5.0 / 6, 0.5, 0, 0}, {0.25, 1.75, 0.75, -1.75, 0}};
        const double At[5][5] = {{0, 0, 0, 0, 0}, {0, 0.5, 0, 0, 0}, {0, 1.0 / 6, 0.5, 0, 0},
                                 {0, -0.5, 0.5, 0.5, 0}, {0, 1.5, -1.5, 0.5, 0.5}};
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < 5; ++j) {
                T.a[i][j] = A[i][j];
                T.at[i][j] = At[i][j];
            }
        const double b[5] = {0.25, 1.75, 0.75, -1.75, 0}, bt[5] = {0, 1.5, -1.5, 0.5, 0.5};
        for (int i = 0; i < 5; ++i) {
            T.b[i] = b[i];
            T.bt[i] = bt[i];
        }
    }
    return T;
}

}  // namespace

cudaError_t launch_imex_rates(hdg_handle *h, const double *u, const double *hh, double *nu, double *nh, double *lu,
                              double *lh) {
    Imex &I = h->imex;
    HDG_DISPATCH_P(h->p, (upwind_trace_kernel<P><<<nblocks(h->NF, 256), 256, 0, h->stream>>>(
                             h->NF, h->d_facet_cell, h->d_facet_edge, h->d_flip, h->d_X, u, hh, h->prm.H, h->tau_s,
                             I.lam)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    RateArgs a{h->N, h->NF, h->prm.g, h->prm.H, h->tau_s, h->d_ref, I.minv, h->d_X, I.fcell, h->d_facet_of,
               h->d_flip, I.lam, u, hh, nu, nh, lu, lh};
    HDG_DISPATCH_P(h->p, (imex_rates_kernel<P><<<nblocks(h->N, 128), 128, 0, h->stream>>>(a)));
    return cudaGetLastError();
}

}  // namespace hdg

using namespace hdg;

namespace {

int imex_fail(hdg_handle *h, int code, const std::string &msg) {
    h->err = msg;
    return code;
}

void imex_free(Imex &I) {
    for (double **p : {&I.fcell, &I.minv, &I.lam, &I.lam_out, &I.buf})
        if (*p) {
            cudaFree(*p);
            *p = nullptr;
        }
    I.ready = false;
}

}  // namespace

void hdg::imex_release(hdg_handle *h) { imex_free(h->imex); }

extern "C" int hdg_imex_init(hdg_handle *h, const double *f_vertex) {
    if (!h) return HDG_EINVAL;
    if (h->prm.flux != 0)
        return imex_fail(h, HDG_EINVAL, "hdg_imex_init: the IMEX stages use the upwind solver");
    if (h->has_f)
        return imex_fail(h, HDG_EINVAL,
                         "hdg_imex_init: the implicit stages have no Coriolis term; set the handle up with "
                         "f_vertex = NULL and pass the Coriolis field here");
    Imex &I = h->imex;
    imex_free(I);
    const size_t N = h->N, np = h->np, nq = N * 3 * np;
    // inverse reference mass matrix (Gauss-Jordan with partial pivoting, host)
    RefElem re = build_ref_elem(h->p);
    const int n = int(np);
    std::vector<double> A(re.M), inv(size_t(n) * n, 0.0);
    for (int i = 0; i < n; ++i) inv[size_t(i) * n + i] = 1.0;
    for (int k = 0; k < n; ++k) {
        int piv = k;
        for (int r = k + 1; r < n; ++r)
            if (std::fabs(A[size_t(r) * n + k]) > std::fabs(A[size_t(piv) * n + k])) piv = r;
        for (int c = 0; c < n; ++c) {
            std::swap(A[size_t(k) * n + c], A[size_t(piv) * n + c]);
            std::swap(inv[size_t(k) * n + c], inv[size_t(piv) * n + c]);
        }
        const double d = 1.0 / A[size_t(k) * n + k];
        for (int c = 0; c < n; ++c) {
            A[size_t(k) * n + c] *= d;
            inv[size_t(k) * n + c] *= d;
        }
        for (int r = 0; r < n; ++r)
            if (r != k) {
                const double f = A[size_t(r) * n + k];
                for (int c = 0; c < n; ++c) {
                    A[size_t(r) * n + c] -= f * A[size_t(k) * n + c];
                    inv[size_t(r) * n + c] -= f * inv[size_t(k) * n + c];
                }
            }
    }
    std::vector<double> fcell(N * 3, 0.0);
    I.has_f = false;
    if (f_vertex)
        for (size_t K = 0; K < N; ++K)
            for (int i = 0; i < 3; ++i) {
                fcell[K * 3 + i] = f_vertex[h->hm.cells[3 * K + i]];
                if (fcell[K * 3 + i] != 0.0) I.has_f = true;
            }
    // state buffers: 3 + 2 * kImexMaxStages state vectors (stage state, stage
    // right-hand side, a copy of q0, the two rates of every stage)
    I.nq = nq;
    const size_t nbuf = size_t(3 + 2 * kImexMaxStages) * nq;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&I.fcell), sizeof(double) * N * 3);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&I.minv), sizeof(double) * np * np);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&I.lam), sizeof(double) * size_t(h->NT));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&I.lam_out), sizeof(double) * size_t(h->NT));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&I.buf), sizeof(double) * nbuf);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(I.fcell, fcell.data(), sizeof(double) * N * 3, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(I.minv, inv.data(), sizeof(double) * np * np, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        imex_free(I);
        return imex_fail(h, e == cudaErrorMemoryAllocation ? HDG_ENOMEM : HDG_ECUDA,
                         std::string("hdg_imex_init: ") + cudaGetErrorString(e));
    }
    I.ready = true;
    return HDG_OK;
}

extern "C" int hdg_imex_rates_dev(hdg_handle *h, const double *u, const double *hh, double *nu, double *nh,
                                  double *lu, double *lh) {
    if (!h) return HDG_EINVAL;
    if (!h->imex.ready) return imex_fail(h, HDG_ESTATE, "hdg_imex_init has not run on this handle");
    if (!u || !hh || !lu || !lh || (!nu) != (!nh)) return imex_fail(h, HDG_EINVAL, "NULL pointer argument");
    cudaError_t e = account_launch(h, HDG_PROF_IMEX, 2, [&]() { return launch_imex_rates(h, u, hh, nu, nh, lu, lh); });
    if (e != cudaSuccess) return imex_fail(h, HDG_ECUDA, std::string("hdg_imex_rates_dev: ") + cudaGetErrorString(e));
    return HDG_OK;
}

extern "C" int hdg_imex_step_dev(hdg_handle *h, int scheme, double theta, double dt, double *u, double *hh,
                                 hdg_solve_info *info) {
    if (!h) return HDG_EINVAL;
    Imex &I = h->imex;
    if (!I.ready) return imex_fail(h, HDG_ESTATE, "hdg_imex_init has not run on this handle");
    if (!u || !hh) return imex_fail(h, HDG_EINVAL, "NULL pointer argument");
    if (scheme < HDG_IMEX_THETA || scheme > HDG_IMEX_ARS3) return imex_fail(h, HDG_EINVAL, "unknown IMEX scheme");
    if (!(dt > 0)) return imex_fail(h, HDG_EINVAL, "dt must be positive");
    if (scheme == HDG_IMEX_THETA && !(theta > 0 && theta <= 1))
        return imex_fail(h, HDG_EINVAL, "theta must be in (0, 1]");
    const Tableau T = tableau(scheme, theta);
    // every implicit stage of these schemes has the same a~_ii: one operator
    double alpha = 0.0;
    for (int i = 0; i < T.s; ++i)
        if (T.at[i][i] != 0.0) alpha = T.at[i][i];
    const double tau = alpha * dt;
    if (!h->condensed || std::fabs(h->prm.tau - tau) > 1e-15 * tau) {
        const int rc = hdg_set_tau(h, tau);
        if (rc) return rc;
    }
    const size_t nq = I.nq, nu_ = size_t(h->N) * 2 * h->np;
    double *Q = I.buf, *R = I.buf + nq, *q0k = I.buf + 2 * nq;
    double *rn[kImexMaxStages], *rl[kImexMaxStages];
    for (int i = 0; i < kImexMaxStages; ++i) {
        rn[i] = I.buf + (3 + 2 * i) * nq;
        rl[i] = I.buf + (4 + 2 * i) * nq;
    }
    cudaStream_t s = h->stream;
    // q0 as one contiguous state vector (u part, then h part)
    cudaError_t e = cudaMemcpyAsync(q0k, u, sizeof(double) * nu_, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(q0k + nu_, hh, sizeof(double) * (nq - nu_), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return imex_fail(h, HDG_ECUDA, std::string("hdg_imex_step_dev: ") + cudaGetErrorString(e));
    hdg_solve_info acc{};
    int status = HDG_OK;
    const bool expl_f = I.has_f;
    for (int i = 0; i < T.s; ++i) {
        // stage right-hand side r_i = q0 + dt sum_{j<i} (a_ij n~_j + a~_ij l~_j)
        Combo c{};
        c.k = i;
        for (int j = 0; j < i; ++j) {
            c.cn[j] = expl_f ? T.a[i][j] : 0.0;
            c.cl[j] = T.at[i][j];
            c.n[j] = rn[j];
            c.l[j] = rl[j];
        }
        double *Qi;
        if (i == 0 && T.at[0][0] == 0.0) {
            Qi = q0k;                                   // explicit first stage: Q_1 = q0
        } else {
            e = account_launch(h, HDG_PROF_IMEX, 1, [&]() {
                imex_combine_kernel<<<nblocks(nq, 256), 256, 0, s>>>(nq, q0k, c, dt, R);
                return cudaGetLastError();
            });
            if (e != cudaSuccess) return imex_fail(h, HDG_ECUDA, std::string("imex combine: ") + cudaGetErrorString(e));
            if (T.at[i][i] != 0.0) {
                hdg_solve_info si{};
                int rc = hdg_solve_dev(h, R, R + nu_, I.lam_out, &si);
                acc.iters += si.iters;
                acc.outer += si.outer;
                acc.true_rel_res = std::max(acc.true_rel_res, si.true_rel_res);
                acc.est_rel_res = std::max(acc.est_rel_res, si.est_rel_res);
                if (rc && !status) status = rc;
                if (rc == HDG_ECUDA || rc == HDG_ENAN) break;
                // the stage's recovery from what its step 1 kept (two-float handles), else from R
                const bool kz = solve_kept_z(h);
                rc = hdg_recover_dev(h, kz ? nullptr : R, kz ? nullptr : R + nu_, nullptr, Q, Q + nu_);
                if (rc) return rc;
                Qi = Q;
            } else {
                Qi = R;                                 // M Q = M r: a mass solve in function space
            }
        }
        // the stage's rates n~(Q_i), l~(Q_i)
        e = account_launch(h, HDG_PROF_IMEX, 2, [&]() {
            return launch_imex_rates(h, Qi, Qi + nu_, expl_f ? rn[i] : nullptr, expl_f ? rn[i] + nu_ : nullptr,
                                     rl[i], rl[i] + nu_);
        });
        if (e != cudaSuccess) return imex_fail(h, HDG_ECUDA, std::string("imex rates: ") + cudaGetErrorString(e));
    }
    if (status == HDG_ECUDA || status == HDG_ENAN) {
        acc.status = status;
        if (info) *info = acc;
        return status;
    }
    // q1 = q0 + dt sum_i (b_i n~_i + b~_i l~_i), written into the caller's u, h
    Combo c{};
    c.k = T.s;
    for (int j = 0; j < T.s; ++j) {
        c.cn[j] = expl_f ? T.b[j] : 0.0;
        c.cl[j] = T.bt[j];
        c.n[j] = rn[j];
        c.l[j] = rl[j];
    }
    e = account_launch(h, HDG_PROF_IMEX, 1, [&]() {
        imex_combine_kernel<<<nblocks(nq, 256), 256, 0, s>>>(nq, q0k, c, dt, R);
        return cudaGetLastError();
    });
    if (e == cudaSuccess) e = cudaMemcpyAsync(u, R, sizeof(double) * nu_, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hh, R + nu_, sizeof(double) * (nq - nu_), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return imex_fail(h, HDG_ECUDA, std::string("hdg_imex_step_dev: ") + cudaGetErrorString(e));
    acc.status = status;
    if (info) *info = acc;
    return status;
}
