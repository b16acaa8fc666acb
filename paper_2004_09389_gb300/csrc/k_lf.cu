// Lax-Friedrichs HDG variant (flux = 1): vector trace u_hat in [P^p(e)]^2 and
// the lowest-order Raviart-Thomas coarse space (Sec. 4.1 Eq. bilinear_HDG_lax,
// App. B, Sec. 4.4 Eq. coarse_problem_LF), flat periodic meshes, FP64.
//
// Per cell, with the momentum rows scaled by H/g (their symmetric part is then
// diag((H/g)(M + tau tau_s E), (H/g)(M + tau tau_s E), M) and the couplings are
// skew, so Gauss-Jordan elimination needs no pivoting):
//   momentum: (u,w) + tau (f u_perp, w) - tau g (h, div w) + tau g <h, w.n>
//             + tau tau_s <u, w>_dK - tau tau_s <u_hat, w>_dK
//   mass:     (h,psi) - tau H (u, grad psi) + tau H <u_hat.n, psi>_dK
//   facet:    <g h n + tau_s u, w_hat> - tau_s <u_hat, w_hat>
// i.e. A_K q + B_K u_hat = Mass_K r and C_K q - Mt_K u_hat; the outputs are
// those of the upwind condensation (A^-1 B, A^-1 Mass, S_K = Mt + C A^-1 B,
// C A^-1 Mass) with M = 6(p+1) local trace dofs: edge i, component c, node j
// at i * 2(p+1) + c (p+1) + j.  On a facet the trace dofs are component-major,
// nodes from the lower to the higher vertex id, so the facet-row kernels run
// unchanged on blocks of TB = 2(p+1) (the handle's pf = TB - 1).
//
// RT0 (one normal-flux dof per facet, along the facet's global normal nu_e,
// the direction lo -> hi turned clockwise): pi u_c = the average of the two
// cells' RT0 fields at the trace nodes (the L2 projection onto P^p(e) of a
// linear function), restriction pi^T, and the coarse operator
//   S_c = (1/tau) [(u, w) + tau f_K (u_perp, w) + tau^2 g H (div u, div w)]
// (coarse_mode 1 drops the rotation), assembled per ELL slot of the facet
// stencil (the facet and its four neighbours) from per-cell 3 x 3 matrices.
#include "common.h"

#include <cmath>

namespace hdg {

namespace {

inline unsigned nblk(size_t n, int bs) { return unsigned((n + bs - 1) / bs); }

template <int P>
struct SzL {
    static constexpr int PP = P + 1;
    static constexpr int TB = 2 * PP;
    static constexpr int NP = (P + 1) * (P + 2) / 2;
    static constexpr int NK = 3 * NP;
    static constexpr int M = 3 * TB;
    static constexpr int LDA = NK + M + NK;
};

struct CondenseLFArgs {
    int N;
    double tau, g, H, tau_s;
    const double *ref, *X, *fcell;
    double *Xb, *Rm, *W, *Scell;
    int32_t *status;
};

template <int P>
__global__ void __launch_bounds__(128) condense_lf_kernel(CondenseLFArgs a) {
    using S = SzL<P>;
    constexpr int NP = S::NP, NK = S::NK, M = S::M, PP = S::PP, TB = S::TB, LDA = S::LDA;
    constexpr int oM = 0, oML = oM + NP * NP, oDxi = oML + 3 * NP * NP, oDeta = oDxi + NP * NP,
                  oE = oDeta + NP * NP, oN = oE + 3 * NP * NP, oM1 = oN + 3 * NP * PP;
    extern __shared__ double smem[];
    double *Aug = smem;                 // [NK][LDA]
    double *Cm = Aug + NK * LDA;        // [M][NK]
    double *prow = Cm + M * NK;         // [LDA]
    double *fac = prow + LDA;           // [NK]
    __shared__ double geo[16];          // det, Jit[4], len[3], nrm[6]
    __shared__ double fK[3];
    __shared__ int bad;
    const int K = blockIdx.x, tid = threadIdx.x;
    const double *ref = a.ref;
    if (tid == 0) {
        const double *x = a.X + size_t(K) * 6;
        const double J00 = x[2] - x[0], J01 = x[4] - x[0], J10 = x[3] - x[1], J11 = x[5] - x[1];
        const double det = J00 * J11 - J01 * J10;
        geo[0] = det;
        geo[1] = J11 / det; geo[2] = -J10 / det;
        geo[3] = -J01 / det; geo[4] = J00 / det;
        for (int i = 0; i < 3; ++i) {
            const int v1 = (i + 1) % 3, v2 = (i + 2) % 3;
            const double tx = x[2 * v2] - x[2 * v1], ty = x[2 * v2 + 1] - x[2 * v1 + 1];
            const double l = sqrt(tx * tx + ty * ty);
            geo[5 + i] = l;
            geo[8 + 2 * i] = ty / l;
            geo[9 + 2 * i] = -tx / l;
        }
        for (int i = 0; i < 3; ++i) fK[i] = a.fcell[size_t(K) * 3 + i];
        bad = 0;
    }
    __syncthreads();
    const double det = geo[0], j00 = geo[1], j01 = geo[2], j10 = geo[3], j11 = geo[4];
    const double tau = a.tau, g = a.g, H = a.H, ts = a.tau_s, sH = H / g;
    for (int idx = tid; idx < NK * LDA; idx += blockDim.x) {
        const int rho = idx / LDA, col = idx % LDA;
        const int R = rho / NP, ia = rho % NP;
        double v = 0.0;
        if (col < NK) {
            const int Cc = col / NP, ib = col % NP;
            const double Mab = det * ref[oM + ia * NP + ib];
            double e = 0.0;
            for (int i = 0; i < 3; ++i) e += geo[5 + i] * ref[oE + (i * NP + ia) * NP + ib];
            if (R < 2) {
                if (Cc == R) {
                    v = Mab + tau * ts * e;
                } else if (Cc < 2) {
                    const double mf = det * (fK[0] * ref[oML + ia * NP + ib] + fK[1] * ref[oML + NP * NP + ia * NP + ib] +
                                             fK[2] * ref[oML + 2 * NP * NP + ia * NP + ib]);
                    v = (R == 0 ? -tau : tau) * mf;
                } else {
                    // -tau g (h, d_R phi_a) + tau g <h, phi_a n_R>
                    const double dxi = ref[oDxi + ib * NP + ia], deta = ref[oDeta + ib * NP + ia];
                    const double d = (R == 0) ? det * (j00 * dxi + j01 * deta) : det * (j10 * dxi + j11 * deta);
                    double en = 0.0;
                    for (int i = 0; i < 3; ++i) en += geo[5 + i] * geo[8 + 2 * i + R] * ref[oE + (i * NP + ia) * NP + ib];
                    v = -tau * g * d + tau * g * en;
                }
                v *= sH;
            } else {
                if (Cc < 2) {
                    // -tau H (u_Cc, d_Cc psi_a)
                    const double dxi = ref[oDxi + ib * NP + ia], deta = ref[oDeta + ib * NP + ia];
                    const double d = (Cc == 0) ? det * (j00 * dxi + j01 * deta) : det * (j10 * dxi + j11 * deta);
                    v = -tau * H * d;
                } else {
                    v = Mab;
                }
            }
        } else if (col < NK + M) {
            const int t = col - NK, i = t / TB, c = (t / PP) % 2, j = t % PP;
            const double nl = geo[5 + i] * ref[oN + (i * NP + ia) * PP + j];
            if (R < 2) v = (R == c) ? -tau * ts * nl * sH : 0.0;          // -tau tau_s <u_hat, w> (scaled)
            else v = tau * H * geo[8 + 2 * i + c] * nl;                      // tau H <u_hat.n, psi>
        } else {
            const int kap = col - NK - M, Cc = kap / NP, ib = kap % NP;
            if (Cc == R) v = det * ref[oM + ia * NP + ib] * (R < 2 ? sH : 1.0);
        }
        Aug[idx] = v;
    }
    for (int idx = tid; idx < M * NK; idx += blockDim.x) {
        const int t = idx / NK, kap = idx % NK;
        const int i = t / TB, c = (t / PP) % 2, j = t % PP, Cc = kap / NP, ib = kap % NP;
        const double nl = geo[5 + i] * ref[oN + (i * NP + ib) * PP + j];
        Cm[idx] = (Cc == c) ? ts * nl : (Cc == 2) ? g * geo[8 + 2 * i + c] * nl : 0.0;
    }
    __syncthreads();
    for (int k = 0; k < NK; ++k) {
        const double piv = Aug[k * LDA + k];
        if (!(fabs(piv) > 1e-300) && tid == 0) bad = 1;
        const double pinv = 1.0 / piv;
        for (int c = k + 1 + tid; c < LDA; c += blockDim.x) prow[c] = Aug[k * LDA + c] * pinv;
        for (int r = tid; r < NK; r += blockDim.x) fac[r] = Aug[r * LDA + k];
        __syncthreads();
        const int Wd = LDA - k - 1;
        for (int idx = tid; idx < NK * Wd; idx += blockDim.x) {
            const int r = idx / Wd, c = k + 1 + idx % Wd;
            if (r == k) Aug[r * LDA + c] = prow[c];
            else Aug[r * LDA + c] -= fac[r] * prow[c];
        }
        __syncthreads();
    }
    if (bad) {
        if (tid == 0) atomicOr(a.status, 1);
        return;
    }
    const size_t N = a.N;
    for (int idx = tid; idx < NK * M; idx += blockDim.x) {
        const int rho = idx / M, t = idx % M;
        a.Xb[size_t(idx) * N + K] = Aug[rho * LDA + NK + t];
    }
    for (int idx = tid; idx < NK * NK; idx += blockDim.x) {
        const int rho = idx / NK, kap = idx % NK;
        a.Rm[size_t(idx) * N + K] = Aug[rho * LDA + NK + M + kap];
    }
    for (int idx = tid; idx < M * M; idx += blockDim.x) {
        const int t = idx / M, t2 = idx % M;
        double s = 0.0;
        for (int kap = 0; kap < NK; ++kap) s += Cm[t * NK + kap] * Aug[kap * LDA + NK + t2];
        if (t / PP == t2 / PP)               // same edge and component: tau_s <u_hat, w_hat>
            s += ts * geo[5 + t / TB] * ref[oM1 + (t % PP) * PP + (t2 % PP)];
        a.Scell[size_t(K) * M * M + idx] = s;
    }
    for (int idx = tid; idx < M * NK; idx += blockDim.x) {
        const int t = idx / NK, kap = idx % NK;
        double s = 0.0;
        for (int r = 0; r < NK; ++r) s += Cm[t * NK + r] * Aug[r * LDA + NK + M + kap];
        a.W[size_t(idx) * N + K] = s;
    }
}

// facet-row operator and inverted diagonal blocks on TB x TB blocks (the layout
// of the upwind assembly with PP replaced by TB)
struct AssembleLFArgs {
    int NF;
    const double *Scell;
    const int32_t *facet_of, *flip, *facet_cell, *facet_edge;
    double *Sval, *Dinv;
    int32_t *nbr, *status;
};

template <int P>
__device__ __forceinline__ int lf_local(int i, int r, int F) {
    constexpr int PP = P + 1, TB = 2 * PP;
    const int c = r / PP, jj = r % PP;
    return i * TB + c * PP + (F ? P - jj : jj);
}

template <int P>
__global__ void assemble_lf_kernel(AssembleLFArgs a) {
    constexpr int PP = P + 1, TB = 2 * PP, M = 3 * TB;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.NF) return;
    const size_t NF = a.NF;
    int K[2], I[2], F[2];
    for (int s = 0; s < 2; ++s) {
        K[s] = a.facet_cell[2 * e + s];
        I[s] = a.facet_edge[2 * e + s];
        F[s] = a.flip[3 * K[s] + I[s]];
    }
    double D[TB][TB];
    for (int r = 0; r < TB; ++r)
        for (int c = 0; c < TB; ++c) {
            double v = 0.0;
            for (int s = 0; s < 2; ++s)
                v += a.Scell[size_t(K[s]) * M * M + lf_local<P>(I[s], r, F[s]) * M + lf_local<P>(I[s], c, F[s])];
            D[r][c] = v;
            a.Sval[packed_index((r * 5 + 0) * TB + c, e, NF, 2)] = v;
        }
    for (int s = 0; s < 2; ++s)
        for (int k = 0; k < 2; ++k) {
            const int b = 1 + 2 * s + k;
            const int i2 = (I[s] + 1 + k) % 3;
            const int f2 = a.flip[3 * K[s] + i2];
            a.nbr[size_t(b - 1) * NF + e] = a.facet_of[3 * K[s] + i2];
            for (int r = 0; r < TB; ++r)
                for (int c = 0; c < TB; ++c)
                    a.Sval[packed_index((r * 5 + b) * TB + c, e, NF, 2)] =
                        a.Scell[size_t(K[s]) * M * M + lf_local<P>(I[s], r, F[s]) * M + lf_local<P>(i2, c, f2)];
        }
    double Inv[TB][TB];
    for (int r = 0; r < TB; ++r)
        for (int c = 0; c < TB; ++c) Inv[r][c] = (r == c) ? 1.0 : 0.0;
    bool singular = false;
    for (int k = 0; k < TB; ++k) {
        int pr = k;
        double best = fabs(D[k][k]);
        for (int r = k + 1; r < TB; ++r)
            if (fabs(D[r][k]) > best) { best = fabs(D[r][k]); pr = r; }
        if (!(best > 1e-300)) { singular = true; break; }
        if (pr != k)
            for (int c = 0; c < TB; ++c) {
                double t = D[k][c]; D[k][c] = D[pr][c]; D[pr][c] = t;
                t = Inv[k][c]; Inv[k][c] = Inv[pr][c]; Inv[pr][c] = t;
            }
        const double pinv = 1.0 / D[k][k];
        for (int c = 0; c < TB; ++c) { D[k][c] *= pinv; Inv[k][c] *= pinv; }
        for (int r = 0; r < TB; ++r) {
            if (r == k) continue;
            const double f = D[r][k];
            for (int c = 0; c < TB; ++c) { D[r][c] -= f * D[k][c]; Inv[r][c] -= f * Inv[k][c]; }
        }
    }
    if (singular) atomicOr(a.status, 2);
    for (int r = 0; r < TB; ++r)
        for (int c = 0; c < TB; ++c) a.Dinv[packed_index(r * TB + c, e, NF, 2)] = Inv[r][c];
}

// step 1, cell part (M = 6(p+1) rows) and facet gather
template <int P>
__global__ void rhs_cell_lf_kernel(int N, const double *__restrict__ W, const double *__restrict__ r_u,
                                   const double *__restrict__ r_h, double *__restrict__ ycell) {
    constexpr int NP = (P + 1) * (P + 2) / 2, NK = 3 * NP, M = 6 * (P + 1);
    const size_t idx = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= size_t(N) * M) return;
    const int t = int(idx / N), K = int(idx % N);
    double acc = 0.0;
    for (int kap = 0; kap < NK; ++kap) {
        const double rv = kap < 2 * NP ? r_u[size_t(K) * 2 * NP + kap] : r_h[size_t(K) * NP + kap - 2 * NP];
        acc = fma(__ldg(W + size_t(t * NK + kap) * N + K), rv, acc);
    }
    ycell[idx] = acc;
}

template <int P>
__global__ void rhs_gather_lf_kernel(int N, int NF, const double *__restrict__ ycell, const int32_t *__restrict__ fcell,
                                     const int32_t *__restrict__ fedge, const int32_t *__restrict__ flip,
                                     double *__restrict__ g) {
    constexpr int TB = 2 * (P + 1);
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NF) return;
    double v[TB];
    for (int r = 0; r < TB; ++r) v[r] = 0.0;
    for (int s = 0; s < 2; ++s) {
        const int K = fcell[2 * e + s], i = fedge[2 * e + s], f = flip[3 * K + i];
        for (int r = 0; r < TB; ++r) v[r] += ycell[size_t(lf_local<P>(i, r, f)) * N + K];
    }
    for (int r = 0; r < TB; ++r) g[size_t(r) * NF + e] = v[r];
}

// step 3: q_K = R_M r_K - X_B u_hat_K
template <int P>
__global__ void recover_lf_kernel(int N, int NF, const double *__restrict__ Rm, const double *__restrict__ Xb,
                                  const double *__restrict__ r_u, const double *__restrict__ r_h,
                                  const double *__restrict__ lam, const int32_t *__restrict__ facet_of,
                                  const int32_t *__restrict__ flip, double *__restrict__ u, double *__restrict__ hout) {
    constexpr int PP = P + 1, TB = 2 * PP, NP = (P + 1) * (P + 2) / 2, NK = 3 * NP, M = 3 * TB;
    const size_t idx = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= size_t(N) * NK) return;
    const int rho = int(idx / N), K = int(idx % N);
    double acc = 0.0;
    for (int kap = 0; kap < NK; ++kap) {
        const double rv = kap < 2 * NP ? r_u[size_t(K) * 2 * NP + kap] : r_h[size_t(K) * NP + kap - 2 * NP];
        acc = fma(__ldg(Rm + size_t(rho * NK + kap) * N + K), rv, acc);
    }
    for (int i = 0; i < 3; ++i) {
        const int f = facet_of[3 * K + i], fl = flip[3 * K + i];
        for (int c = 0; c < 2; ++c)
            for (int j = 0; j < PP; ++j)
                acc = fma(-__ldg(Xb + size_t(rho * M + i * TB + c * PP + j) * N + K),
                          lam[size_t(c * PP + (fl ? P - j : j)) * NF + f], acc);
    }
    if (rho < 2 * NP) u[size_t(K) * 2 * NP + rho] = acc;
    else hout[size_t(K) * NP + rho - 2 * NP] = acc;
}

// ---------------------------------------------------------------- RT0

// S_c in ELL form Sc[b * NF + f], b = 0 the facet itself, b = 1..4 its neighbours
__global__ void rt0_assemble_kernel(int nslot, const int32_t *__restrict__ ptr, const int32_t *__restrict__ code,
                                    const double *__restrict__ loc, const double *__restrict__ fK, double tau,
                                    double gH, int rotating, double *__restrict__ Sc) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nslot) return;
    double acc = 0.0;
    for (int k = ptr[q]; k < ptr[q + 1]; ++k) {
        const int c = code[k], K = c / 9, ij = c % 9;
        const double *l = loc + size_t(K) * 27;
        const double f = rotating ? fK[K] : 0.0;
        acc += (l[ij] + tau * f * l[9 + ij] + tau * tau * gH * l[18 + ij]) / tau;
    }
    Sc[q] = acc;
}

__global__ void rt0_dinv_kernel(int NF, const double *__restrict__ Sc, double *__restrict__ dinv) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f < NF) dinv[f] = 1.0 / Sc[f];
}

// y = D_c^-1 S_c x (used by the spectral estimate)
__global__ void rt0_apply_dinv_kernel(int NF, const double *__restrict__ Sc, const int32_t *__restrict__ nbr,
                                      const double *__restrict__ dinv, const double *__restrict__ x,
                                      double *__restrict__ y) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= NF) return;
    double acc = Sc[f] * x[f];
    for (int b = 1; b < 5; ++b) acc = fma(Sc[size_t(b) * NF + f], x[nbr[size_t(b - 1) * NF + f]], acc);
    y[f] = dinv[f] * acc;
}

// a step of the Chebyshev iteration on S_c e = r (x null: the previous iterate
// is zero; xprev null likewise): out = x + omega D_c^-1 (r - S_c x) + beta (x - xprev)
__global__ void rt0_cheb_kernel(int NF, const double *__restrict__ Sc, const int32_t *__restrict__ nbr,
                                const double *__restrict__ dinv, const double *__restrict__ r, const double *x,
                                const double *xprev, double *out, double omega, double beta) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= NF) return;
    double res = r[f];
    double xf = 0.0;
    if (x) {
        xf = x[f];
        res -= Sc[f] * xf;
        for (int b = 1; b < 5; ++b) res = fma(-Sc[size_t(b) * NF + f], x[nbr[size_t(b - 1) * NF + f]], res);
    }
    const double xp = xprev ? xprev[f] : 0.0;
    out[f] = xf + omega * dinv[f] * res + beta * (xf - xp);
}

// r_c = pi^T r: coarse dof f gathers from the trace dofs of itself and of its
// four neighbours e (the block of e whose neighbour is f: rev)
template <int P>
__global__ void rt0_restrict_kernel(int NF, const int32_t *__restrict__ nbr, const int32_t *__restrict__ rev,
                                    const double *__restrict__ piw, const double *__restrict__ r,
                                    double *__restrict__ rc) {
    constexpr int TB = 2 * (P + 1);
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= NF) return;
    double acc = 0.0;
    for (int q = 0; q < TB; ++q) acc = fma(piw[size_t(q) * NF + f], r[size_t(q) * NF + f], acc);
    for (int bp = 1; bp < 5; ++bp) {
        const int e = nbr[size_t(bp - 1) * NF + f], b = rev[size_t(bp - 1) * NF + f];
        for (int q = 0; q < TB; ++q) acc = fma(piw[size_t(b * TB + q) * NF + e], r[size_t(q) * NF + e], acc);
    }
    rc[f] = acc;
}

// x += pi e_c
template <int P>
__global__ void rt0_prolong_add_kernel(int NF, const int32_t *__restrict__ nbr, const double *__restrict__ piw,
                                       const double *__restrict__ ec, double *__restrict__ x) {
    constexpr int TB = 2 * (P + 1);
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NF) return;
    double c[5];
    c[0] = ec[e];
    for (int b = 1; b < 5; ++b) c[b] = ec[nbr[size_t(b - 1) * NF + e]];
    for (int q = 0; q < TB; ++q) {
        double acc = x[size_t(q) * NF + e];
        for (int b = 0; b < 5; ++b) acc = fma(piw[size_t(b * TB + q) * NF + e], c[b], acc);
        x[size_t(q) * NF + e] = acc;
    }
}

}  // namespace

// ---------------------------------------------------------------- host set-up of RT0

std::string build_rt0(const HostMesh &hm, int p, Rt0Host &o) {
    const int NF = hm.nf, N = hm.nc, PP = p + 1, TB = 2 * PP;
    o = Rt0Host();
    // facet-row neighbours, as the facet-row assembly orders them
    o.nbr.assign(size_t(4) * NF, 0);
    for (int e = 0; e < NF; ++e)
        for (int s = 0; s < 2; ++s) {
            const int K = hm.facet_cell[2 * e + s], I = hm.facet_edge[2 * e + s];
            for (int k = 0; k < 2; ++k) o.nbr[size_t(2 * s + k) * NF + e] = hm.facet_of[3 * K + (I + 1 + k) % 3];
        }
    auto nb = [&](int e, int b) { return b == 0 ? e : o.nbr[size_t(b - 1) * NF + e]; };
    for (int e = 0; e < NF; ++e)
        for (int b = 0; b < 5; ++b)
            for (int b2 = b + 1; b2 < 5; ++b2)
                if (nb(e, b) == nb(e, b2)) return "Lax-Friedrichs solver: a facet stencil repeats a facet (mesh too small)";
    // global facet normals nu_e (from the first cell of each facet) and cell signs
    std::vector<double> nu(size_t(2) * NF);
    auto cellX = [&](int K, int v, int d) { return hm.X[size_t(K) * 6 + v * 2 + d]; };
    for (int e = 0; e < NF; ++e) {
        const int K = hm.facet_cell[2 * e], I = hm.facet_edge[2 * e];
        const int a = (I + 1) % 3, b = (I + 2) % 3;
        double tx = cellX(K, b, 0) - cellX(K, a, 0), ty = cellX(K, b, 1) - cellX(K, a, 1);
        if (hm.flip[3 * K + I]) { tx = -tx; ty = -ty; }
        const double l = std::sqrt(tx * tx + ty * ty);
        nu[2 * size_t(e)] = ty / l;
        nu[2 * size_t(e) + 1] = -tx / l;
    }
    std::vector<double> sig(size_t(3) * N), len(size_t(3) * N), det(N);
    for (int K = 0; K < N; ++K) {
        const double J00 = cellX(K, 1, 0) - cellX(K, 0, 0), J01 = cellX(K, 2, 0) - cellX(K, 0, 0);
        const double J10 = cellX(K, 1, 1) - cellX(K, 0, 1), J11 = cellX(K, 2, 1) - cellX(K, 0, 1);
        det[size_t(K)] = J00 * J11 - J01 * J10;
        for (int i = 0; i < 3; ++i) {
            const int a = (i + 1) % 3, b = (i + 2) % 3;
            const double tx = cellX(K, b, 0) - cellX(K, a, 0), ty = cellX(K, b, 1) - cellX(K, a, 1);
            const double l = std::sqrt(tx * tx + ty * ty);
            len[3 * size_t(K) + i] = l;
            const int f = hm.facet_of[3 * K + i];
            sig[3 * size_t(K) + i] = (ty / l) * nu[2 * size_t(f)] + (-tx / l) * nu[2 * size_t(f) + 1] > 0 ? 1.0 : -1.0;
        }
    }
    // RT0 basis of local edge i of K at x: |e_i| / det (x - X_i), times the sign
    auto phi = [&](int K, int i, double x, double y, double &vx, double &vy) {
        const double s = sig[3 * size_t(K) + i] * len[3 * size_t(K) + i] / det[size_t(K)];
        vx = s * (x - cellX(K, i, 0));
        vy = s * (y - cellX(K, i, 1));
    };
    // prolongation weights piw[(b TB + c PP + jj) NF + e]
    o.piw.assign(size_t(5) * TB * NF, 0.0);
    for (int e = 0; e < NF; ++e)
        for (int s = 0; s < 2; ++s) {
            const int K = hm.facet_cell[2 * e + s], I = hm.facet_edge[2 * e + s], F = hm.flip[3 * K + I];
            const int a = (I + 1) % 3, b = (I + 2) % 3;
            for (int jj = 0; jj < PP; ++jj) {
                const double t = F ? 1.0 - double(jj) / p : double(jj) / p;
                const double x = cellX(K, a, 0) + t * (cellX(K, b, 0) - cellX(K, a, 0));
                const double y = cellX(K, a, 1) + t * (cellX(K, b, 1) - cellX(K, a, 1));
                for (int i2 = 0; i2 < 3; ++i2) {
                    const int blk = (i2 == I) ? 0 : 1 + 2 * s + (i2 - I - 1 + 3) % 3;
                    double vx, vy;
                    phi(K, i2, x, y, vx, vy);
                    o.piw[(size_t(blk * TB + 0 * PP + jj)) * NF + e] += 0.5 * vx;
                    o.piw[(size_t(blk * TB + 1 * PP + jj)) * NF + e] += 0.5 * vy;
                }
            }
        }
    // rev[(b' - 1) NF + f]: the block b of e = nbr_b'(f) whose facet is f
    o.rev.assign(size_t(4) * NF, -1);
    for (int f = 0; f < NF; ++f)
        for (int bp = 1; bp < 5; ++bp) {
            const int e = nb(f, bp);
            for (int b = 1; b < 5; ++b)
                if (nb(e, b) == f) o.rev[size_t(bp - 1) * NF + f] = b;
            if (o.rev[size_t(bp - 1) * NF + f] < 0) return "Lax-Friedrichs solver: facet stencil is not symmetric";
        }
    // per-cell 3 x 3 matrices [M | R | D] (test i, trial j; global signs) and the slot lists
    o.loc.assign(size_t(27) * N, 0.0);
    o.fK.assign(size_t(N), 0.0);
    std::vector<std::vector<int32_t>> slots(size_t(5) * NF);
    for (int K = 0; K < N; ++K) {
        const double area = 0.5 * det[size_t(K)];
        double px[3][3], py[3][3];   // basis i at edge midpoint k
        for (int k = 0; k < 3; ++k) {
            const int a = (k + 1) % 3, b = (k + 2) % 3;
            const double x = 0.5 * (cellX(K, a, 0) + cellX(K, b, 0)), y = 0.5 * (cellX(K, a, 1) + cellX(K, b, 1));
            for (int i = 0; i < 3; ++i) phi(K, i, x, y, px[i][k], py[i][k]);
        }
        double *l = &o.loc[size_t(27) * K];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double m = 0.0, r = 0.0;
                for (int k = 0; k < 3; ++k) {
                    m += px[i][k] * px[j][k] + py[i][k] * py[j][k];
                    r += px[i][k] * (-py[j][k]) + py[i][k] * px[j][k];     // phi_i . phi_j_perp
                }
                const double di = sig[3 * size_t(K) + i] * len[3 * size_t(K) + i] / area;
                const double dj = sig[3 * size_t(K) + j] * len[3 * size_t(K) + j] / area;
                l[i * 3 + j] = area / 3.0 * m;
                l[9 + i * 3 + j] = area / 3.0 * r;
                l[18 + i * 3 + j] = area * di * dj;
                const int fi = hm.facet_of[3 * K + i], fj = hm.facet_of[3 * K + j];
                int slot = -1;
                for (int b = 0; b < 5; ++b)
                    if (nb(fi, b) == fj) slot = b;
                if (slot < 0) return "Lax-Friedrichs solver: RT0 coupling outside the facet stencil";
                slots[size_t(slot) * NF + fi].push_back(K * 9 + i * 3 + j);
            }
    }
    o.ptr.assign(slots.size() + 1, 0);
    for (size_t q = 0; q < slots.size(); ++q) {
        o.ptr[q + 1] = o.ptr[q] + int32_t(slots[q].size());
        o.code.insert(o.code.end(), slots[q].begin(), slots[q].end());
    }
    return "";
}

// ---------------------------------------------------------------- launchers

cudaError_t launch_condense_lf(hdg_handle *h) {
    auto run = [&](auto tag) -> cudaError_t {
        constexpr int P = decltype(tag)::value;
        using S = SzL<P>;
        const size_t smem = sizeof(double) * (S::NK * S::LDA + S::M * S::NK + S::LDA + S::NK);
        cudaError_t e = cudaFuncSetAttribute(condense_lf_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(smem));
        if (e != cudaSuccess) return e;
        CondenseLFArgs a{h->N, h->prm.tau, h->prm.g, h->prm.H, h->tau_s, h->d_ref, h->d_X, h->d_fcell,
                         h->d_Xb, h->d_Rm, h->d_W, h->d_Scell, h->d_status};
        condense_lf_kernel<P><<<h->N, 128, smem, h->stream>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        AssembleLFArgs b{h->NF, h->d_Scell, h->d_facet_of, h->d_flip, h->d_facet_cell, h->d_facet_edge,
                         h->d_Sval, h->d_Dinv, h->d_nbr, h->d_status};
        assemble_lf_kernel<P><<<nblk(h->NF, 128), 128, 0, h->stream>>>(b);
        return cudaGetLastError();
    };
    switch (h->p) {
        case 1: return run(std::integral_constant<int, 1>());
        case 2: return run(std::integral_constant<int, 2>());
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_rhs_lf(hdg_handle *h, const double *r_u, const double *r_h, double *g, double *ycell) {
    const size_t n = size_t(h->N) * h->m;
    switch (h->p) {
        case 1:
            rhs_cell_lf_kernel<1><<<nblk(n, 256), 256, 0, h->stream>>>(h->N, h->d_W, r_u, r_h, ycell);
            rhs_gather_lf_kernel<1><<<nblk(h->NF, 256), 256, 0, h->stream>>>(h->N, h->NF, ycell, h->d_facet_cell,
                                                                             h->d_facet_edge, h->d_flip, g);
            break;
        case 2:
            rhs_cell_lf_kernel<2><<<nblk(n, 256), 256, 0, h->stream>>>(h->N, h->d_W, r_u, r_h, ycell);
            rhs_gather_lf_kernel<2><<<nblk(h->NF, 256), 256, 0, h->stream>>>(h->N, h->NF, ycell, h->d_facet_cell,
                                                                             h->d_facet_edge, h->d_flip, g);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_recover_lf(hdg_handle *h, const double *r_u, const double *r_h, const double *lam, double *u,
                              double *hout) {
    const size_t n = size_t(h->N) * h->nK;
    switch (h->p) {
        case 1:
            recover_lf_kernel<1><<<nblk(n, 256), 256, 0, h->stream>>>(h->N, h->NF, h->d_Rm, h->d_Xb, r_u, r_h, lam,
                                                                       h->d_facet_of, h->d_flip, u, hout);
            break;
        case 2:
            recover_lf_kernel<2><<<nblk(n, 256), 256, 0, h->stream>>>(h->N, h->NF, h->d_Rm, h->d_Xb, r_u, r_h, lam,
                                                                       h->d_facet_of, h->d_flip, u, hout);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_rt0_assemble(hdg_handle *h) {
    const Rt0Dev &R = h->rt0;
    const int nslot = 5 * h->NF;
    rt0_assemble_kernel<<<nblk(nslot, 256), 256, 0, h->stream>>>(nslot, R.ptr, R.code, R.loc, R.fK, h->prm.tau,
                                                                 h->prm.g * h->prm.H, h->prm.coarse_mode == 0 ? 1 : 0,
                                                                 R.Sc);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    rt0_dinv_kernel<<<nblk(h->NF, 256), 256, 0, h->stream>>>(h->NF, R.Sc, R.dinv);
    return cudaGetLastError();
}

cudaError_t launch_rt0_apply_dinv(hdg_handle *h, const double *x, double *y) {
    rt0_apply_dinv_kernel<<<nblk(h->NF, 256), 256, 0, h->stream>>>(h->NF, h->rt0.Sc, h->rt0.nbr, h->rt0.dinv, x, y);
    return cudaGetLastError();
}

cudaError_t launch_rt0_cheb(hdg_handle *h, const double *r, const double *x, const double *xprev, double *out,
                            double omega, double beta) {
    rt0_cheb_kernel<<<nblk(h->NF, 256), 256, 0, h->stream>>>(h->NF, h->rt0.Sc, h->rt0.nbr, h->rt0.dinv, r, x, xprev,
                                                             out, omega, beta);
    return cudaGetLastError();
}

cudaError_t launch_rt0_restrict(hdg_handle *h, const double *r, double *rc) {
    const Rt0Dev &R = h->rt0;
    switch (h->p) {
        case 1: rt0_restrict_kernel<1><<<nblk(h->NF, 256), 256, 0, h->stream>>>(h->NF, R.nbr, R.rev, R.piw, r, rc); break;
        case 2: rt0_restrict_kernel<2><<<nblk(h->NF, 256), 256, 0, h->stream>>>(h->NF, R.nbr, R.rev, R.piw, r, rc); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_rt0_prolong_add(hdg_handle *h, const double *ec, double *x) {
    const Rt0Dev &R = h->rt0;
    switch (h->p) {
        case 1: rt0_prolong_add_kernel<1><<<nblk(h->NF, 256), 256, 0, h->stream>>>(h->NF, R.nbr, R.piw, ec, x); break;
        case 2: rt0_prolong_add_kernel<2><<<nblk(h->NF, 256), 256, 0, h->stream>>>(h->NF, R.nbr, R.piw, ec, x); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace hdg
