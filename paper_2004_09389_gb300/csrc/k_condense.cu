// Static condensation (Sec. 4.2) and assembly of the facet-row trace operator.
//
// Per cell K (one CTA per cell), with u_perp = (-u_y, u_x), the cell rows of
// the upwind HDG form (Eq. bilinear_HDG_upwind, ABCM split of Eq. ABCMform /
// App. B, Coriolis implicit) are assembled in the integrated-by-parts form
//   momentum: (u,w) + tau (f u_perp, w) - tau g (h, div w)         + tau g <lambda, w.n>
//   mass:     (h,psi) + tau H (div u, psi) + tau tau_s <h, psi>_dK - tau tau_s <lambda, psi>
//   facet:    <H u.n + tau_s h, mu> - tau_s <lambda, mu>
// i.e. A_K q + B_K lambda = Mass_K r on the cell and C_K q - Mt_K lambda on its
// facets.  The momentum rows are scaled by H/g: the scaled A_K has the
// positive-definite symmetric part  diag((H/g) M, M + tau tau_s E)  (the
// Coriolis and the tau H div coupling are skew after scaling), so every
// leading minor is non-zero and Gauss-Jordan elimination needs no pivoting.
// Elimination of [A | B | Mass] gives X_B = A^-1 B and R_M = A^-1 Mass; then
//   S_K = Mt_K + C_K X_B      (the cell's part of Eq. schur_system)
//   W_K = C_K R_M             (step 1: g = sum_K P_K^T W_K r_K)
// and R_M, X_B serve step 3 (Eq. reconstruct_solution): q = R_M r - X_B lambda_K.
#include "common.h"

#include <cstdlib>

namespace hdg {

namespace {

constexpr int kCondenseThreads = 128;

template <int P>
struct Sz {
    static constexpr int PP = P + 1;
    static constexpr int NP = (P + 1) * (P + 2) / 2;
    static constexpr int NK = 3 * NP;
    static constexpr int M = 3 * PP;
    static constexpr int LDA = NK + M + NK;
};

struct CondenseArgs {
    int N;
    double tau, g, H, tau_s;
    const double *ref;      // packed reference matrices
    const double *X;        // [N][3][2]
    const double *fcell;    // [N][3]
    double *Xb, *Rm, *W, *Scell;
    int32_t *status;
    float4 *Xb2, *Rm2, *W2;   // mixed-precision kernel: the float-pair copies, written directly
};

// The cell's system in shared memory: geometry (geo: detJ, J^-T, edge
// lengths, outward normals), the vertex Coriolis values fK, the augmented rows
// [D A | D B | D Mass] (Aug, NK x LDA; D the momentum-row scaling) and C (Cm,
// M x NK).  Ends with a barrier.
template <int P>
__device__ __forceinline__ void cell_system(const CondenseArgs &a, int K, double *Aug, double *Cm, double *geo,
                                            double *fK) {
    using S = Sz<P>;
    constexpr int NP = S::NP, NK = S::NK, M = S::M, PP = S::PP, LDA = S::LDA;
    constexpr int oM = 0, oML = oM + NP * NP, oDxi = oML + 3 * NP * NP, oDeta = oDxi + NP * NP,
                  oE = oDeta + NP * NP, oN = oE + 3 * NP * NP;
    const int tid = threadIdx.x;
    const double *ref = a.ref;
    if (tid == 0) {
        const double *x = a.X + size_t(K) * 6;
        double J00 = x[2] - x[0], J01 = x[4] - x[0], J10 = x[3] - x[1], J11 = x[5] - x[1];
        double det = J00 * J11 - J01 * J10;
        geo[0] = det;
        // Jit = J^-T
        geo[1] = J11 / det;  geo[2] = -J10 / det;
        geo[3] = -J01 / det; geo[4] = J00 / det;
        for (int i = 0; i < 3; ++i) {
            int v1 = (i + 1) % 3, v2 = (i + 2) % 3;
            double tx = x[2 * v2] - x[2 * v1], ty = x[2 * v2 + 1] - x[2 * v1 + 1];
            double l = sqrt(tx * tx + ty * ty);
            geo[5 + i] = l;
            geo[8 + 2 * i] = ty / l;       // outward normal of a counter-clockwise cell
            geo[9 + 2 * i] = -tx / l;
        }
        for (int i = 0; i < 3; ++i) fK[i] = a.fcell[size_t(K) * 3 + i];
    }
    __syncthreads();
    const double det = geo[0], j00 = geo[1], j01 = geo[2], j10 = geo[3], j11 = geo[4];
    const double tau = a.tau, g = a.g, H = a.H, ts = a.tau_s, sH = H / g;

    // ---- assemble [D A | D B | D Mass] and C
    for (int idx = tid; idx < NK * LDA; idx += blockDim.x) {
        const int rho = idx / LDA, col = idx % LDA;
        const int R = rho / NP, ia = rho % NP;
        double v = 0.0;
        if (col < NK) {
            const int Cc = col / NP, ib = col % NP;
            const double Mab = det * ref[oM + ia * NP + ib];
            if (R < 2) {
                if (Cc == R) v = Mab;
                else if (Cc < 2) {
                    double mf = det * (fK[0] * ref[oML + ia * NP + ib] + fK[1] * ref[oML + NP * NP + ia * NP + ib] +
                                       fK[2] * ref[oML + 2 * NP * NP + ia * NP + ib]);
                    v = (R == 0 ? -tau : tau) * mf;
                } else {
                    // -tau g (h, d_x phi_a): D_x[b][a] = int phi_b d_x phi_a
                    double dxi = ref[oDxi + ib * NP + ia], deta = ref[oDeta + ib * NP + ia];
                    double d = (R == 0) ? det * (j00 * dxi + j01 * deta) : det * (j10 * dxi + j11 * deta);
                    v = -tau * g * d;
                }
                v *= sH;
            } else {
                if (Cc < 2) {
                    // tau H (d_x u_x, psi_a): D_x[a][b]
                    double dxi = ref[oDxi + ia * NP + ib], deta = ref[oDeta + ia * NP + ib];
                    double d = (Cc == 0) ? det * (j00 * dxi + j01 * deta) : det * (j10 * dxi + j11 * deta);
                    v = tau * H * d;
                } else {
                    double e = 0.0;
                    for (int i = 0; i < 3; ++i) e += geo[5 + i] * ref[oE + (i * NP + ia) * NP + ib];
                    v = Mab + tau * ts * e;
                }
            }
        } else if (col < NK + M) {
            const int t = col - NK, i = t / PP, j = t % PP;
            const double nl = geo[5 + i] * ref[oN + (i * NP + ia) * PP + j];
            if (R == 0) v = tau * H * geo[8 + 2 * i] * nl;        // (H/g) tau g n_x <lambda, phi_a>
            else if (R == 1) v = tau * H * geo[9 + 2 * i] * nl;
            else v = -tau * ts * nl;
        } else {
            const int kap = col - NK - M, Cc = kap / NP, ib = kap % NP;
            if (Cc == R) v = det * ref[oM + ia * NP + ib] * (R < 2 ? sH : 1.0);
        }
        Aug[idx] = v;
    }
    for (int idx = tid; idx < M * NK; idx += blockDim.x) {
        const int t = idx / NK, kap = idx % NK;
        const int i = t / PP, j = t % PP, Cc = kap / NP, ib = kap % NP;
        const double nl = geo[5 + i] * ref[oN + (i * NP + ib) * PP + j];
        Cm[idx] = (Cc == 0) ? H * geo[8 + 2 * i] * nl : (Cc == 1) ? H * geo[9 + 2 * i] * nl : ts * nl;
    }
    __syncthreads();

}

template <int P>
__global__ void __launch_bounds__(kCondenseThreads) condense_kernel(CondenseArgs a) {
    using S = Sz<P>;
    constexpr int NP = S::NP, NK = S::NK, M = S::M, PP = S::PP, LDA = S::LDA;
    constexpr int oM = 0, oML = oM + NP * NP, oDxi = oML + 3 * NP * NP, oDeta = oDxi + NP * NP,
                  oE = oDeta + NP * NP, oN = oE + 3 * NP * NP, oM1 = oN + 3 * NP * PP;
    extern __shared__ double smem[];
    double *Aug = smem;                 // [NK][LDA]
    double *Cm = Aug + NK * LDA;        // [M][NK]
    double *prow = Cm + M * NK;         // [LDA]
    double *fac = prow + LDA;           // [NK]
    __shared__ double geo[16];          // detJ, Jit[4], len[3], nrm[6], pad
    __shared__ double fK[3];
    __shared__ int bad;

    const int K = blockIdx.x;
    const int tid = threadIdx.x;
    const double *ref = a.ref;
    const double ts = a.tau_s;
    if (tid == 0) bad = 0;
    cell_system<P>(a, K, Aug, Cm, geo, fK);

    // ---- Gauss-Jordan elimination, no pivoting (see the header comment)
    for (int k = 0; k < NK; ++k) {
        const double piv = Aug[k * LDA + k];
        if (!(fabs(piv) > 1e-300)) {
            if (tid == 0) bad = 1;
        }
        const double pinv = 1.0 / piv;
        for (int c = k + 1 + tid; c < LDA; c += blockDim.x) prow[c] = Aug[k * LDA + c] * pinv;
        for (int r = tid; r < NK; r += blockDim.x) fac[r] = Aug[r * LDA + k];
        __syncthreads();
        const int W = LDA - k - 1;
        for (int idx = tid; idx < NK * W; idx += blockDim.x) {
            const int r = idx / W, c = k + 1 + idx % W;
            if (r == k) Aug[r * LDA + c] = prow[c];
            else Aug[r * LDA + c] -= fac[r] * prow[c];
        }
        __syncthreads();
    }
    if (bad) {
        if (tid == 0) atomicOr(a.status, 1);
        return;
    }

    // ---- outputs
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
        if (t / PP == t2 / PP)
            s += ts * geo[5 + t / PP] * ref[oM1 + (t % PP) * PP + (t2 % PP)];
        a.Scell[size_t(K) * M * M + idx] = s;
    }
    for (int idx = tid; idx < M * NK; idx += blockDim.x) {
        const int t = idx / NK, kap = idx % NK;
        double s = 0.0;
        for (int r = 0; r < NK; ++r) s += Cm[t * NK + r] * Aug[r * LDA + NK + M + kap];
        a.W[size_t(idx) * N + K] = s;
    }
}

// ---------------------------------------------------------------- mixed-precision condensation
// The same outputs for the mixed-precision handles, which use X_B, R_M, S_K
// and W_K only as two-float pairs (and FP32 / BF16 copies): A_K is inverted in
// FP32 (Gauss-Jordan in place, no pivoting, as above), X = A^-1 [B | Mass]
// formed in FP32 and refined twice, each time with the residual
// [B | Mass] - A X formed in two-float arithmetic (FFAcc) from the FP64 system
// and the two-float X, and the correction A^-1 R added to X, kept as a
// two-float pair.  S_K = Mt_K + C X_B and W_K = C R_M are formed in two-float
// arithmetic too.  Each refinement step gains the factor ||I - Ainv A|| (about
// cond(A_K) 2^-24) up to the two-float resolution (about 2^-48 relative):
// two steps reach it for cells with a condition number well below 2^12.  No
// FP64 product or elimination is left (GB300's FP32 rate is about 70 times its
// FP64 rate), and with an explicit FP32 inverse every solve is a product, free
// of the barrier per elimination step that triangular solves would take.
// refinement steps (each costs about 60 % of the kernel's instructions)
constexpr int kMpRefine = 2;

template <int P>
struct SzMp {
    using S = Sz<P>;
    static constexpr int NR = S::M + S::NK;                        // right-hand sides: B, Mass
    static constexpr int oAi = S::NK * S::LDA + S::M * S::NK;      // in doubles: after Aug and Cm
    static constexpr int nAi = (S::NK * S::NK + 1) / 2;            // FP32 inverse
    static constexpr int oAp = oAi + nAi;                          // split A (float2 = one double each)
    static constexpr int oXp = oAp + S::NK * S::NK;                // two-float X
    static constexpr int oBp = oXp + S::NK * NR;                   // split right-hand sides
    static constexpr int oRf = oBp + S::NK * NR;                   // FP32 residual
    static constexpr int oFac = oRf + (S::NK * NR + 1) / 2;        // FP32 column factors
    static constexpr int total = oFac + (S::NK + 1) / 2;           // doubles of dynamic shared memory
};

template <int P>
__global__ void __launch_bounds__(kCondenseThreads) condense_mp_kernel(CondenseArgs a) {
    using S = Sz<P>;
    using Z = SzMp<P>;
    constexpr int NP = S::NP, NK = S::NK, M = S::M, PP = S::PP, LDA = S::LDA, NR = Z::NR;
    constexpr int oM1 = NP * NP + 3 * NP * NP + NP * NP + NP * NP + 3 * NP * NP + 3 * NP * PP;
    extern __shared__ double smem[];
    double *Aug = smem;                                            // [NK][LDA]
    double *Cm = Aug + NK * LDA;                                   // [M][NK]
    float *Ai = reinterpret_cast<float *>(smem + Z::oAi);          // [NK][NK] FP32 inverse
    float2 *Ap = reinterpret_cast<float2 *>(smem + Z::oAp);        // [NK][NK] split A; later split C
    float2 *Xp = reinterpret_cast<float2 *>(smem + Z::oXp);        // [NK][NR] two-float X
    float2 *Bp = reinterpret_cast<float2 *>(smem + Z::oBp);        // [NK][NR] split [B | Mass]
    float *Rf = reinterpret_cast<float *>(smem + Z::oRf);          // [NK][NR]
    float *fac = reinterpret_cast<float *>(smem + Z::oFac);        // [NK]
    __shared__ double geo[16];
    __shared__ double fK[3];
    __shared__ int bad;

    const int K = blockIdx.x;
    const int tid = threadIdx.x;
    const double *ref = a.ref;
    const double ts = a.tau_s;
    if (tid == 0) bad = 0;
    cell_system<P>(a, K, Aug, Cm, geo, fK);

    for (int idx = tid; idx < NK * NK; idx += blockDim.x) {
        const float2 v = split(Aug[(idx / NK) * LDA + idx % NK]);
        Ap[idx] = v;
        Ai[idx] = v.x;
    }
    __syncthreads();
    // ---- FP32 inverse in place: step k scales row k (its pivot entry becomes
    // 1 / pivot) and records column k, then eliminates column k from the other
    // rows (their column-k entries become -a_ik / pivot)
    for (int k = 0; k < NK; ++k) {
        const float piv = Ai[k * NK + k];
        if (tid == 0 && !(fabsf(piv) > 1e-30f)) bad = 1;
        const float pinv = 1.0f / piv;
        for (int i = tid; i < NK; i += blockDim.x) fac[i] = Ai[i * NK + k];
        __syncthreads();
        for (int c = tid; c < NK; c += blockDim.x) Ai[k * NK + c] = (c == k) ? pinv : Ai[k * NK + c] * pinv;
        __syncthreads();
        for (int idx = tid; idx < NK * NK; idx += blockDim.x) {
            const int i = idx / NK, c = idx % NK;
            if (i == k) continue;
            Ai[idx] = (c == k) ? -fac[i] * pinv : fmaf(-fac[i], Ai[k * NK + c], Ai[idx]);
        }
        __syncthreads();
    }
    if (bad) {
        if (tid == 0) atomicOr(a.status, 1);
        return;
    }
    // ---- X_0 = Ainv [B | Mass] in FP32, then the refinement steps
    for (int idx = tid; idx < NK * NR; idx += blockDim.x) {
        const float2 v = split(Aug[(idx / NR) * LDA + NK + idx % NR]);
        Bp[idx] = v;
        Rf[idx] = v.x;
    }
    __syncthreads();
    for (int idx = tid; idx < NK * NR; idx += blockDim.x) {
        const int i = idx / NR, c = idx % NR;
        float x = 0.0f;
#pragma unroll 6
        for (int j = 0; j < NK; ++j) x = fmaf(Ai[i * NK + j], Rf[j * NR + c], x);
        Xp[idx] = make_float2(x, 0.0f);
    }
    __syncthreads();
    for (int it = 0; it < kMpRefine; ++it) {
        for (int idx = tid; idx < NK * NR; idx += blockDim.x) {
            const int r = idx / NR, c = idx % NR;
            FFAcc acc;
#pragma unroll 5
            for (int j = 0; j < NK; ++j) acc.add(Ap[r * NK + j], Xp[j * NR + c]);
            // r = b - A X to FP32 accuracy: the leading parts nearly cancel exactly
            const float2 bv = Bp[idx];
            Rf[idx] = __fadd_rn(__fsub_rn(bv.x, acc.s), __fsub_rn(bv.y, acc.c));
        }
        __syncthreads();
        for (int idx = tid; idx < NK * NR; idx += blockDim.x) {
            const int i = idx / NR, c = idx % NR;
            float d = 0.0f;
#pragma unroll 6
            for (int j = 0; j < NK; ++j) d = fmaf(Ai[i * NK + j], Rf[j * NR + c], d);
            // (hi, lo) + d: TwoSum of the leading parts, then renormalise
            const float2 x = Xp[idx];
            const float s1 = __fadd_rn(x.x, d);
            const float bp = __fsub_rn(s1, x.x);
            const float e = __fadd_rn(__fsub_rn(x.x, __fsub_rn(s1, bp)), __fsub_rn(d, bp));
            const float lo = __fadd_rn(x.y, e);
            const float hi = __fadd_rn(s1, lo);
            Xp[idx] = make_float2(hi, __fsub_rn(lo, __fsub_rn(hi, s1)));
        }
        __syncthreads();
    }
    // ---- outputs: X_B, R_M and W_K as float pairs in the cell tiles of the
    // two-float kernels, S_K in FP64 (C split into the space of the split A)
    float2 *Cp = Ap;
    for (int idx = tid; idx < M * NK; idx += blockDim.x) Cp[idx] = split(Cm[idx]);
    __syncthreads();
    {
        constexpr int CPb = (M + 1) / 2, CPr = (NK + 1) / 2;
        for (int idx = tid; idx < NK * CPb; idx += blockDim.x) {
            const int rho = idx / CPb, c0 = 2 * (idx % CPb);
            const float2 x0 = Xp[rho * NR + c0];
            const float2 x1 = c0 + 1 < M ? Xp[rho * NR + c0 + 1] : make_float2(0.f, 0.f);
            a.Xb2[ff_pair_index(size_t(K), size_t(idx), size_t(NK) * CPb)] = make_float4(x0.x, x0.y, x1.x, x1.y);
        }
        for (int idx = tid; idx < NK * CPr; idx += blockDim.x) {
            const int rho = idx / CPr, c0 = 2 * (idx % CPr);
            const float2 x0 = Xp[rho * NR + M + c0];
            const float2 x1 = c0 + 1 < NK ? Xp[rho * NR + M + c0 + 1] : make_float2(0.f, 0.f);
            a.Rm2[ff_pair_index(size_t(K), size_t(idx), size_t(NK) * CPr)] = make_float4(x0.x, x0.y, x1.x, x1.y);
        }
        // W_K = C R_M: each pair of columns from two two-float sums, renormalised
        for (int idx = tid; idx < M * CPr; idx += blockDim.x) {
            const int t = idx / CPr, c0 = 2 * (idx % CPr);
            float v[4] = {0.f, 0.f, 0.f, 0.f};
            for (int q = 0; q < 2 && c0 + q < NK; ++q) {
                FFAcc acc;
                for (int r = 0; r < NK; ++r) acc.add(Cp[t * NK + r], Xp[r * NR + M + c0 + q]);
                const float hi = __fadd_rn(acc.s, acc.c);
                v[2 * q] = hi;
                v[2 * q + 1] = __fsub_rn(acc.c, __fsub_rn(hi, acc.s));
            }
            a.W2[ff_pair_index(size_t(K), size_t(idx), size_t(M) * CPr)] = make_float4(v[0], v[1], v[2], v[3]);
        }
    }
    for (int idx = tid; idx < M * M; idx += blockDim.x) {
        const int t = idx / M, t2 = idx % M;
        FFAcc acc;
        for (int kap = 0; kap < NK; ++kap) acc.add(Cp[t * NK + kap], Xp[kap * NR + t2]);
        double v = acc.value();
        if (t / PP == t2 / PP) v += ts * geo[5 + t / PP] * ref[oM1 + (t % PP) * PP + (t2 % PP)];
        a.Scell[size_t(K) * M * M + idx] = v;
    }
}

// ---------------------------------------------------------------- facet-row assembly
// For facet e with incident (cell, local edge) pairs (K_s, i_s), s = 0, 1, row r
// of the facet (trace node r from the lower to the higher vertex id) is
//   (S x)_{e,r} = sum_c D_e[r][c] x_{e,c} + sum_{s,k} O_{s,k}[r][c] x_{nbr(s,k),c}
// with D_e the sum of both cells' diagonal blocks and O_{s,k} the block of S_{K_s}
// coupling edge i_s to edge (i_s + 1 + k) % 3 (neighbour facet nbr(s,k)).
// Element j = (r*5 + b)*PP + c (b = 0: D_e, b = 1 + 2s + k) of facet e is stored at
// packed_index(j, e, NF, 2) (16-byte groups of two doubles); Dinv = D_e^-1 likewise.
// Padding lanes of the last group are zero.
struct AssembleArgs {
    int N, NF;
    const double *Scell;
    const int32_t *facet_of, *flip, *facet_cell, *facet_edge;
    double *Sval, *Dinv;
    int32_t *nbr;
    int32_t *status;
};

template <int P>
__global__ void assemble_kernel(AssembleArgs a) {
    constexpr int PP = P + 1, M = 3 * PP;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.NF) return;
    const size_t NF = a.NF;
    int K[2], I[2], F[2];
    for (int s = 0; s < 2; ++s) {
        K[s] = a.facet_cell[2 * e + s];
        I[s] = a.facet_edge[2 * e + s];
        F[s] = a.flip[3 * K[s] + I[s]];
    }
    double D[PP][PP];
    for (int r = 0; r < PP; ++r)
        for (int c = 0; c < PP; ++c) {
            double v = 0.0;
            for (int s = 0; s < 2; ++s) {
                const int lr = I[s] * PP + (F[s] ? P - r : r);
                const int lc = I[s] * PP + (F[s] ? P - c : c);
                v += a.Scell[size_t(K[s]) * M * M + lr * M + lc];
            }
            D[r][c] = v;
            a.Sval[packed_index((r * 5 + 0) * PP + c, e, NF, 2)] = v;
        }
    for (int s = 0; s < 2; ++s)
        for (int k = 0; k < 2; ++k) {
            const int b = 1 + 2 * s + k;
            const int i2 = (I[s] + 1 + k) % 3;
            const int f2 = a.flip[3 * K[s] + i2];
            a.nbr[size_t(b - 1) * NF + e] = a.facet_of[3 * K[s] + i2];
            for (int r = 0; r < PP; ++r) {
                const int lr = I[s] * PP + (F[s] ? P - r : r);
                for (int c = 0; c < PP; ++c) {
                    const int lc = i2 * PP + (f2 ? P - c : c);
                    a.Sval[packed_index((r * 5 + b) * PP + c, e, NF, 2)] = a.Scell[size_t(K[s]) * M * M + lr * M + lc];
                }
            }
        }
    // invert D_e (Gauss-Jordan with partial pivoting, in registers)
    double Inv[PP][PP];
    for (int r = 0; r < PP; ++r)
        for (int c = 0; c < PP; ++c) Inv[r][c] = (r == c) ? 1.0 : 0.0;
    bool singular = false;
    for (int k = 0; k < PP; ++k) {
        int pr = k;
        double best = fabs(D[k][k]);
        for (int r = k + 1; r < PP; ++r)
            if (fabs(D[r][k]) > best) { best = fabs(D[r][k]); pr = r; }
        if (!(best > 1e-300)) { singular = true; break; }
        if (pr != k)
            for (int c = 0; c < PP; ++c) {
                double t = D[k][c]; D[k][c] = D[pr][c]; D[pr][c] = t;
                t = Inv[k][c]; Inv[k][c] = Inv[pr][c]; Inv[pr][c] = t;
            }
        const double pinv = 1.0 / D[k][k];
        for (int c = 0; c < PP; ++c) { D[k][c] *= pinv; Inv[k][c] *= pinv; }
        for (int r = 0; r < PP; ++r) {
            if (r == k) continue;
            const double f = D[r][k];
            for (int c = 0; c < PP; ++c) { D[r][c] -= f * D[k][c]; Inv[r][c] -= f * Inv[k][c]; }
        }
    }
    if (singular) atomicOr(a.status, 2);
    for (int r = 0; r < PP; ++r)
        for (int c = 0; c < PP; ++c) a.Dinv[packed_index(r * PP + c, e, NF, 2)] = Inv[r][c];
    if ((5 * PP * PP) % 2) a.Sval[packed_index(5 * PP * PP, e, NF, 2)] = 0.0;
    if ((PP * PP) % 2) a.Dinv[packed_index(PP * PP, e, NF, 2)] = 0.0;
}

// ---------------------------------------------------------------- P1 level operator
// The coarse problem obtained, as in Sec. 4.4 (Eq. coarse_problem_upwind), by
// eliminating u from the time-implicit continuum equations, here with the
// Coriolis term implicit: u = (I - tau f J)(r_u - tau g grad h)/(1 + tau^2 f^2),
// hence per cell (f_K the cell mean of f, kappa_K = 1/(1 + tau^2 f_K^2))
//   A = [ (phi,psi) + tau^2 g H kappa_K ((grad phi, grad psi) - tau f_K (J grad phi, grad psi)) ] / tau,
// divided by tau to match the scale of the trace operator on smooth traces.
// rotating = 0 drops f (the form printed in the paper).  Every CSR entry sums
// its contributions in a fixed (cell) order.
__global__ void p1_assemble_kernel(int nnz, const int32_t *__restrict__ cptr, const int32_t *__restrict__ contrib,
                                   const double *__restrict__ elem, const double *__restrict__ fK, double tau,
                                   double gH, int rotating, double *__restrict__ A) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nnz) return;
    double acc = 0.0;
    for (int k = cptr[q]; k < cptr[q + 1]; ++k) {
        const int code = contrib[k], K = code / 9, ab = code % 9;
        const double *el = elem + size_t(K) * 27;
        const double f = rotating ? fK[K] : 0.0;
        const double kap = 1.0 / (1.0 + tau * tau * f * f);
        acc += (el[ab] + tau * tau * gH * kap * (el[9 + ab] - tau * f * el[18 + ab])) / tau;
    }
    A[q] = acc;
}

__global__ void p1_dinv_kernel(int nv, const int32_t *__restrict__ diag, const double *__restrict__ A,
                               double *__restrict__ dinv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nv) dinv[i] = 1.0 / A[diag[i]];
}

// dense copy of a padded ELL matrix (n <= 1024; unused slots add 0 to the
// diagonal), then in-place Gauss-Jordan inverse with partial pivoting by one CTA.
__global__ void ell_to_dense_kernel(int n, int width, const int32_t *col, const double *A, double *D) {
    const int r = blockIdx.x;
    for (int c = threadIdx.x; c < n; c += blockDim.x) D[size_t(r) * n + c] = 0.0;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int q = 0; q < width; ++q) D[size_t(r) * n + col[size_t(r) * width + q]] += A[size_t(r) * width + q];
}

__global__ void dense_inverse_kernel(int n, double *Aw, double *inv, int32_t *status) {
    // Aw: working copy [n][n], destroyed; inv: output [n][n]
    __shared__ int piv_row;
    __shared__ double red_v[1024];
    __shared__ int red_i[1024];
    const int tid = threadIdx.x;
    for (int idx = tid; idx < n * n; idx += blockDim.x) inv[idx] = (idx / n == idx % n) ? 1.0 : 0.0;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        double best = -1.0;
        int bi = k;
        for (int r = k + tid; r < n; r += blockDim.x) {
            double v = fabs(Aw[size_t(r) * n + k]);
            if (v > best) { best = v; bi = r; }
        }
        red_v[tid] = best;
        red_i[tid] = bi;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (tid < s && red_v[tid + s] > red_v[tid]) { red_v[tid] = red_v[tid + s]; red_i[tid] = red_i[tid + s]; }
            __syncthreads();
        }
        if (tid == 0) {
            piv_row = red_i[0];
            if (!(red_v[0] > 1e-300)) atomicOr(status, 4);
        }
        __syncthreads();
        const int pr = piv_row;
        if (pr != k)
            for (int c = tid; c < n; c += blockDim.x) {
                double t = Aw[size_t(k) * n + c]; Aw[size_t(k) * n + c] = Aw[size_t(pr) * n + c]; Aw[size_t(pr) * n + c] = t;
                t = inv[size_t(k) * n + c]; inv[size_t(k) * n + c] = inv[size_t(pr) * n + c]; inv[size_t(pr) * n + c] = t;
            }
        __syncthreads();
        const double pinv = 1.0 / Aw[size_t(k) * n + k];
        __syncthreads();
        for (int c = tid; c < n; c += blockDim.x) {
            Aw[size_t(k) * n + c] *= pinv;
            inv[size_t(k) * n + c] *= pinv;
        }
        __syncthreads();
        for (int idx = tid; idx < n * n; idx += blockDim.x) {
            const int r = idx / n, c = idx % n;
            if (r == k) continue;
            const double f = Aw[size_t(r) * n + k];
            if (c != k) Aw[size_t(r) * n + c] -= f * Aw[size_t(k) * n + c];
            inv[size_t(r) * n + c] -= f * inv[size_t(k) * n + c];
        }
        __syncthreads();
        for (int r = tid; r < n; r += blockDim.x)
            if (r != k) Aw[size_t(r) * n + k] = 0.0;
        __syncthreads();
    }
}

// The same elimination over many blocks, for coarsest levels too large for
// one CTA: step k is two launches, the pivot (search as above, row swap,
// scaling of row k, and a copy of column k as the row factors) and the
// update of every other row, each element with the single-CTA kernel's
// arithmetic, so that both give the same inverse bit for bit.
__global__ void gj_pivot_kernel(int n, int k, double *Aw, double *inv, double *fac, int32_t *status) {
    __shared__ int piv_row;
    __shared__ double red_v[1024];
    __shared__ int red_i[1024];
    const int tid = threadIdx.x;
    double best = -1.0;
    int bi = k;
    for (int r = k + tid; r < n; r += blockDim.x) {
        const double v = fabs(Aw[size_t(r) * n + k]);
        if (v > best) { best = v; bi = r; }
    }
    red_v[tid] = best;
    red_i[tid] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (tid < s && red_v[tid + s] > red_v[tid]) { red_v[tid] = red_v[tid + s]; red_i[tid] = red_i[tid + s]; }
        __syncthreads();
    }
    if (tid == 0) {
        piv_row = red_i[0];
        if (!(red_v[0] > 1e-300)) atomicOr(status, 4);
    }
    __syncthreads();
    const int pr = piv_row;
    if (pr != k)
        for (int c = tid; c < n; c += blockDim.x) {
            double t = Aw[size_t(k) * n + c]; Aw[size_t(k) * n + c] = Aw[size_t(pr) * n + c]; Aw[size_t(pr) * n + c] = t;
            t = inv[size_t(k) * n + c]; inv[size_t(k) * n + c] = inv[size_t(pr) * n + c]; inv[size_t(pr) * n + c] = t;
        }
    __syncthreads();
    const double pinv = 1.0 / Aw[size_t(k) * n + k];
    __syncthreads();
    for (int c = tid; c < n; c += blockDim.x) {
        Aw[size_t(k) * n + c] *= pinv;
        inv[size_t(k) * n + c] *= pinv;
    }
    for (int r = tid; r < n; r += blockDim.x) fac[r] = Aw[size_t(r) * n + k];
}

// (columns left of the pivot of the working copy are skipped: their row-k
// entries are exact zeros, so the single-CTA update leaves them unchanged)
__global__ void gj_update_kernel(int n, int k, double *Aw, double *inv, const double *fac) {
    const size_t idx = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= size_t(n) * n) return;
    const int r = int(idx / n), c = int(idx % n);
    if (r == k) return;
    const double f = fac[r];
    if (c > k) Aw[size_t(r) * n + c] -= f * Aw[size_t(k) * n + c];
    else if (c == k) Aw[size_t(r) * n + k] = 0.0;
    inv[size_t(r) * n + c] -= f * inv[size_t(k) * n + c];
}

__global__ void identity_kernel(int n, double *inv) {
    const size_t idx = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx < size_t(n) * n) inv[idx] = (idx / n == idx % n) ? 1.0 : 0.0;
}

__global__ void to_f32_kernel(const double *x, float *y, size_t n) {
    size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) y[i] = float(x[i]);
}

template <int P>
cudaError_t condense_p(hdg_handle *h) {
    using S = Sz<P>;
    size_t smem = sizeof(double) * (S::NK * S::LDA + S::M * S::NK + S::LDA + S::NK);
    cudaError_t e = cudaFuncSetAttribute(condense_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    CondenseArgs a;
    a.N = h->N; a.tau = h->prm.tau; a.g = h->prm.g; a.H = h->prm.H; a.tau_s = h->tau_s;
    a.ref = h->d_ref; a.X = h->d_X; a.fcell = h->d_fcell;
    a.Xb = h->d_Xb; a.Rm = h->d_Rm; a.W = h->d_W; a.Scell = h->d_Scell; a.status = h->d_status;
    condense_kernel<P><<<h->N, kCondenseThreads, smem, h->stream>>>(a);
    return cudaGetLastError();
}

template <int P>
cudaError_t condense_mp_p(hdg_handle *h) {
    const size_t smem = sizeof(double) * SzMp<P>::total;
    cudaError_t e = cudaFuncSetAttribute(condense_mp_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    CondenseArgs a;
    a.N = h->N; a.tau = h->prm.tau; a.g = h->prm.g; a.H = h->prm.H; a.tau_s = h->tau_s;
    a.ref = h->d_ref; a.X = h->d_X; a.fcell = h->d_fcell;
    a.Xb = h->d_Xb; a.Rm = h->d_Rm; a.W = h->d_W; a.Scell = h->d_Scell; a.status = h->d_status;
    a.Xb2 = reinterpret_cast<float4 *>(h->d_Xb2);
    a.Rm2 = reinterpret_cast<float4 *>(h->d_Rm2);
    a.W2 = reinterpret_cast<float4 *>(h->d_W2);
    if (!a.Xb2 || !a.Rm2 || !a.W2) return cudaErrorInvalidValue;
    condense_mp_kernel<P><<<h->N, kCondenseThreads, smem, h->stream>>>(a);
    return cudaGetLastError();
}

template <int P>
cudaError_t assemble_p(hdg_handle *h) {
    AssembleArgs a;
    a.N = h->N; a.NF = h->NF; a.Scell = h->d_Scell;
    a.facet_of = h->d_facet_of; a.flip = h->d_flip; a.facet_cell = h->d_facet_cell; a.facet_edge = h->d_facet_edge;
    a.Sval = h->d_Sval; a.Dinv = h->d_Dinv; a.nbr = h->d_nbr; a.status = h->d_status;
    assemble_kernel<P><<<(h->NF + 127) / 128, 128, 0, h->stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

namespace {
// HDG_CONDENSE_FP64=1: the FP64 elimination for the mixed handles too (read once)
bool force_fp64_condense() {
    static const bool on = [] {
        const char *e = std::getenv("HDG_CONDENSE_FP64");
        return e && e[0] == '1';
    }();
    return on;
}
}  // namespace

bool condense_writes_pairs(const hdg_handle *h) { return mode_ff(h->prm) && !force_fp64_condense(); }

cudaError_t launch_condense(hdg_handle *h) {
    // mixed-precision handles: FP32 inverse with two-float refinement, writing
    // the float-pair matrices directly
    if (condense_writes_pairs(h)) {
        switch (h->p) {
            case 1: return condense_mp_p<1>(h);
            case 2: return condense_mp_p<2>(h);
            case 3: return condense_mp_p<3>(h);
            case 4: return condense_mp_p<4>(h);
        }
        return cudaErrorInvalidValue;
    }
    switch (h->p) {
        case 1: return condense_p<1>(h);
        case 2: return condense_p<2>(h);
        case 3: return condense_p<3>(h);
        case 4: return condense_p<4>(h);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_assemble(hdg_handle *h) {
    switch (h->p) {
        case 1: return assemble_p<1>(h);
        case 2: return assemble_p<2>(h);
        case 3: return assemble_p<3>(h);
        case 4: return assemble_p<4>(h);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_p1_assemble(hdg_handle *h, DevLevel &L, double tau, double gH, int rotating) {
    p1_assemble_kernel<<<(L.nnz + 255) / 256, 256, 0, h->stream>>>(L.nnz, L.contrib_ptr, L.contrib, L.elem, L.fK, tau,
                                                                    gH, rotating, L.A);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    p1_dinv_kernel<<<(L.nv + 255) / 256, 256, 0, h->stream>>>(L.nv, L.diag, L.A, L.dinv);
    return cudaGetLastError();
}

cudaError_t launch_dense_inverse(hdg_handle *h, const DevLevel &L, double *work, double *inv, int n) {
    ell_to_dense_kernel<<<n, 128, 0, h->stream>>>(n, L.width, L.col, L.A, work);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (n <= 256) {
        dense_inverse_kernel<<<1, 1024, 0, h->stream>>>(n, work, inv, h->d_status);
        return cudaGetLastError();
    }
    // larger coarsest levels: one pivot and one update launch per column, the
    // row factors of each column in their own array
    double *fac = h->d_coarse_fac;
    if (!fac) return cudaErrorInvalidValue;
    const size_t nn = size_t(n) * n;
    const unsigned nb = unsigned((nn + 255) / 256);
    identity_kernel<<<nb, 256, 0, h->stream>>>(n, inv);
    for (int k = 0; k < n; ++k) {
        gj_pivot_kernel<<<1, 1024, 0, h->stream>>>(n, k, work, inv, fac, h->d_status);
        gj_update_kernel<<<nb, 256, 0, h->stream>>>(n, k, work, inv, fac);
    }
    return cudaGetLastError();
}

cudaError_t launch_to_f32(const double *x, float *y, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    to_f32_kernel<<<unsigned((n + 255) / 256), 256, 0, s>>>(x, y, n);
    return cudaGetLastError();
}

}  // namespace hdg
