// Trace-space kernels: the facet-row trace operator and everything that lives
// on the facets.
//
// Internal trace vectors are stored node-major, x[r * NF + e] (node r of facet
// e), so that every thread (one facet) reads and writes coalesced planes.  The
// caller-facing lambda layout [NF][p+1] is converted at the API boundary.
//
// Trace operator (Eq. schur_system): one thread per facet e computes its p+1
// rows  y_{e,r} = sum_{b<5} sum_c Sval[(r*5+b)*PP+c][e] x_{src(b),c}  with
// src(0) = e and src(b) = nbr[b-1][e]: the diagonal block (both cells' S_K
// summed) and the four blocks that couple e to the other two facets of each of
// its cells.  The block-Jacobi smoother (the smoother of Alg. twolevel_vcycle,
// with the facet blocks inverted exactly) is the same pass followed by
//   x_new = x + omega D_e^-1 (b - S x)  on the facet's p+1 values.
#include "common.h"

namespace hdg {

namespace {

template <int P, typename T>
__device__ __forceinline__ void facet_rows(const T *__restrict__ Sval, const int32_t *__restrict__ nbr,
                                           const T *__restrict__ x, int e, size_t NF, T (&y)[P + 1]) {
    constexpr int PP = P + 1;
    int src[5];
    src[0] = e;
#pragma unroll
    for (int b = 1; b < 5; ++b) src[b] = __ldg(nbr + size_t(b - 1) * NF + e);
    T xs[5][PP];
#pragma unroll
    for (int b = 0; b < 5; ++b)
#pragma unroll
        for (int c = 0; c < PP; ++c) xs[b][c] = x[size_t(c) * NF + src[b]];
#pragma unroll
    for (int r = 0; r < PP; ++r) {
        T acc = T(0);
#pragma unroll
        for (int b = 0; b < 5; ++b)
#pragma unroll
            for (int c = 0; c < PP; ++c) acc = fma(__ldg(Sval + size_t((r * 5 + b) * PP + c) * NF + e), xs[b][c], acc);
        y[r] = acc;
    }
}

template <int P, typename T>
__global__ void __launch_bounds__(256) apply_kernel(int NF, const T *__restrict__ Sval, const int32_t *__restrict__ nbr,
                                                    const T *__restrict__ x, T *__restrict__ y) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NF) return;
    T v[P + 1];
    facet_rows<P, T>(Sval, nbr, x, e, NF, v);
#pragma unroll
    for (int r = 0; r <= P; ++r) y[size_t(r) * NF + e] = v[r];
}

template <int P, typename T>
__global__ void __launch_bounds__(256) residual_kernel(int NF, const T *__restrict__ Sval,
                                                       const int32_t *__restrict__ nbr, const T *__restrict__ b,
                                                       const T *__restrict__ x, T *__restrict__ res) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NF) return;
    T v[P + 1];
    facet_rows<P, T>(Sval, nbr, x, e, NF, v);
#pragma unroll
    for (int r = 0; r <= P; ++r) res[size_t(r) * NF + e] = b[size_t(r) * NF + e] - v[r];
}

template <int P, typename T>
__global__ void __launch_bounds__(256) smooth_kernel(int NF, const T *__restrict__ Sval, const T *__restrict__ Dinv,
                                                     const int32_t *__restrict__ nbr, const T *__restrict__ b,
                                                     const T *__restrict__ x, T *__restrict__ xout, T omega) {
    constexpr int PP = P + 1;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NF) return;
    T v[PP];
    facet_rows<P, T>(Sval, nbr, x, e, NF, v);
#pragma unroll
    for (int r = 0; r < PP; ++r) v[r] = b[size_t(r) * NF + e] - v[r];
#pragma unroll
    for (int r = 0; r < PP; ++r) {
        T acc = T(0);
#pragma unroll
        for (int c = 0; c < PP; ++c) acc = fma(__ldg(Dinv + size_t(r * PP + c) * NF + e), v[c], acc);
        xout[size_t(r) * NF + e] = fma(omega, acc, x[size_t(r) * NF + e]);
    }
}

// first sweep from a zero initial guess: x = omega D^-1 b
template <int P, typename T>
__global__ void smooth_first_kernel(int NF, const T *__restrict__ Dinv, const T *__restrict__ b, T *__restrict__ xout,
                                    T omega) {
    constexpr int PP = P + 1;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NF) return;
    T v[PP];
#pragma unroll
    for (int c = 0; c < PP; ++c) v[c] = b[size_t(c) * NF + e];
#pragma unroll
    for (int r = 0; r < PP; ++r) {
        T acc = T(0);
#pragma unroll
        for (int c = 0; c < PP; ++c) acc = fma(__ldg(Dinv + size_t(r * PP + c) * NF + e), v[c], acc);
        xout[size_t(r) * NF + e] = omega * acc;
    }
}

// lambda layout [NF][PP] <-> internal [PP][NF]
__global__ void to_internal_kernel(int NF, int PP, const double *ext, double *in) {
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= size_t(NF) * PP) return;
    const size_t e = i / PP, r = i % PP;
    in[r * NF + e] = ext[i];
}
__global__ void to_external_kernel(int NF, int PP, const double *in, double *ext) {
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= size_t(NF) * PP) return;
    const size_t e = i / PP, r = i % PP;
    ext[i] = in[r * NF + e];
}

// cell unknown kappa of cell K from the caller's r_u [N][2][NP], r_h [N][NP]
template <int NP>
__device__ __forceinline__ double cell_rhs(const double *r_u, const double *r_h, int K, int kap) {
    return kap < 2 * NP ? r_u[size_t(K) * 2 * NP + kap] : r_h[size_t(K) * NP + kap - 2 * NP];
}

// step 1, cell part: ycell[t][K] = sum_kappa W[t*NK + kappa][K] r_K[kappa]
template <int P>
__global__ void rhs_cell_kernel(int N, const double *__restrict__ W, const double *__restrict__ r_u,
                                const double *__restrict__ r_h, double *__restrict__ ycell) {
    constexpr int PP = P + 1, NP = (P + 1) * (P + 2) / 2, NK = 3 * NP, M = 3 * PP;
    const size_t idx = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= size_t(N) * M) return;
    const int t = int(idx / N), K = int(idx % N);
    double acc = 0.0;
#pragma unroll 5
    for (int kap = 0; kap < NK; ++kap)
        acc = fma(__ldg(W + size_t(t * NK + kap) * N + K), cell_rhs<NP>(r_u, r_h, K, kap), acc);
    ycell[idx] = acc;
}

// step 1, facet part: g_{e,r} = sum over the two cells of their row of edge i_s
template <int P>
__global__ void rhs_gather_kernel(int N, int NF, const double *__restrict__ ycell, const int32_t *__restrict__ fcell,
                                  const int32_t *__restrict__ fedge, const int32_t *__restrict__ flip,
                                  double *__restrict__ g) {
    constexpr int PP = P + 1;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NF) return;
    double v[PP];
#pragma unroll
    for (int r = 0; r < PP; ++r) v[r] = 0.0;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int K = fcell[2 * e + s], i = fedge[2 * e + s], f = flip[3 * K + i];
#pragma unroll
        for (int r = 0; r < PP; ++r) v[r] += ycell[size_t(i * PP + (f ? P - r : r)) * N + K];
    }
#pragma unroll
    for (int r = 0; r < PP; ++r) g[size_t(r) * NF + e] = v[r];
}

// step 3: q_K = R_M r_K - X_B lambda_K, written in the caller's u / h layout
template <int P>
__global__ void recover_kernel(int N, int NF, const double *__restrict__ Rm, const double *__restrict__ Xb,
                               const double *__restrict__ r_u, const double *__restrict__ r_h,
                               const double *__restrict__ lam, const int32_t *__restrict__ facet_of,
                               const int32_t *__restrict__ flip, double *__restrict__ u, double *__restrict__ hout) {
    constexpr int PP = P + 1, NP = (P + 1) * (P + 2) / 2, NK = 3 * NP, M = 3 * PP;
    const size_t idx = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= size_t(N) * NK) return;
    const int rho = int(idx / N), K = int(idx % N);
    double acc = 0.0;
#pragma unroll 5
    for (int kap = 0; kap < NK; ++kap)
        acc = fma(__ldg(Rm + size_t(rho * NK + kap) * N + K), cell_rhs<NP>(r_u, r_h, K, kap), acc);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int f = facet_of[3 * K + i], fl = flip[3 * K + i];
#pragma unroll
        for (int j = 0; j < PP; ++j)
            acc = fma(-__ldg(Xb + size_t(rho * M + i * PP + j) * N + K), lam[size_t(fl ? P - j : j) * NF + f], acc);
    }
    if (rho < 2 * NP) u[size_t(K) * 2 * NP + rho] = acc;
    else hout[size_t(K) * NP + rho - 2 * NP] = acc;
}

// P1 restriction rho = pi^T: r_c[v] = sum over facet ends at v of the nodal
// weights of the linear interpolant (1 - t_r at the lower vertex, t_r at the higher)
template <int P, typename T>
__global__ void restrict_kernel(int nv, int NF, const int32_t *__restrict__ v2f_ptr, const int32_t *__restrict__ v2f,
                                const T *__restrict__ r, T *__restrict__ rc) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    T acc = T(0);
    for (int k = v2f_ptr[v]; k < v2f_ptr[v + 1]; ++k) {
        const int code = v2f[k], e = code >> 1, hi = code & 1;
#pragma unroll
        for (int j = 0; j <= P; ++j) {
            const T t = T(j) / T(P);
            acc = fma(hi ? t : T(1) - t, r[size_t(j) * NF + e], acc);
        }
    }
    rc[v] = acc;
}

// x += pi e_c (linear interpolation along each facet)
template <int P, typename T>
__global__ void prolong_add_kernel(int NF, const int32_t *__restrict__ fverts, const T *__restrict__ ec,
                                   T *__restrict__ x) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NF) return;
    const T a = ec[fverts[2 * e]], b = ec[fverts[2 * e + 1]];
#pragma unroll
    for (int j = 0; j <= P; ++j) {
        const T t = T(j) / T(P);
        x[size_t(j) * NF + e] += (T(1) - t) * a + t * b;
    }
}

inline unsigned blocks(size_t n, int bs) { return unsigned((n + bs - 1) / bs); }

#define HDG_DISPATCH_P(p, CALL) \
    switch (p) {                \
        case 1: { constexpr int P = 1; CALL; } break; \
        case 2: { constexpr int P = 2; CALL; } break; \
        case 3: { constexpr int P = 3; CALL; } break; \
        case 4: { constexpr int P = 4; CALL; } break; \
        default: return cudaErrorInvalidValue;        \
    }

}  // namespace

template <typename T>
static const T *sval_of(hdg_handle *h);
template <>
const double *sval_of<double>(hdg_handle *h) { return h->d_Sval; }
template <>
const float *sval_of<float>(hdg_handle *h) { return h->d_Sval32; }
template <typename T>
static const T *dinv_of(hdg_handle *h);
template <>
const double *dinv_of<double>(hdg_handle *h) { return h->d_Dinv; }
template <>
const float *dinv_of<float>(hdg_handle *h) { return h->d_Dinv32; }

template <typename T>
cudaError_t launch_apply_t(hdg_handle *h, const T *x, T *y) {
    HDG_DISPATCH_P(h->p, (apply_kernel<P, T><<<blocks(h->NF, 256), 256, 0, h->stream>>>(h->NF, sval_of<T>(h), h->d_nbr, x, y)));
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_residual_t(hdg_handle *h, const T *b, const T *x, T *r) {
    HDG_DISPATCH_P(h->p, (residual_kernel<P, T><<<blocks(h->NF, 256), 256, 0, h->stream>>>(h->NF, sval_of<T>(h), h->d_nbr, b, x, r)));
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_smooth_t(hdg_handle *h, const T *b, const T *x, T *xout) {
    const T om = T(h->prm.omega);
    HDG_DISPATCH_P(h->p, (smooth_kernel<P, T><<<blocks(h->NF, 256), 256, 0, h->stream>>>(h->NF, sval_of<T>(h), dinv_of<T>(h), h->d_nbr, b, x, xout, om)));
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_smooth_first_t(hdg_handle *h, const T *b, T *x) {
    const T om = T(h->prm.omega);
    HDG_DISPATCH_P(h->p, (smooth_first_kernel<P, T><<<blocks(h->NF, 256), 256, 0, h->stream>>>(h->NF, dinv_of<T>(h), b, x, om)));
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_restrict_t(hdg_handle *h, const T *r, T *rc) {
    HDG_DISPATCH_P(h->p, (restrict_kernel<P, T><<<blocks(h->nv, 256), 256, 0, h->stream>>>(h->nv, h->NF, h->d_v2f_ptr, h->d_v2f, r, rc)));
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_prolong_add_t(hdg_handle *h, const T *ec, T *x) {
    HDG_DISPATCH_P(h->p, (prolong_add_kernel<P, T><<<blocks(h->NF, 256), 256, 0, h->stream>>>(h->NF, h->d_facet_verts, ec, x)));
    return cudaGetLastError();
}

template cudaError_t launch_apply_t<double>(hdg_handle *, const double *, double *);
template cudaError_t launch_apply_t<float>(hdg_handle *, const float *, float *);
template cudaError_t launch_residual_t<double>(hdg_handle *, const double *, const double *, double *);
template cudaError_t launch_residual_t<float>(hdg_handle *, const float *, const float *, float *);
template cudaError_t launch_smooth_t<double>(hdg_handle *, const double *, const double *, double *);
template cudaError_t launch_smooth_t<float>(hdg_handle *, const float *, const float *, float *);
template cudaError_t launch_smooth_first_t<double>(hdg_handle *, const double *, double *);
template cudaError_t launch_smooth_first_t<float>(hdg_handle *, const float *, float *);
template cudaError_t launch_restrict_t<double>(hdg_handle *, const double *, double *);
template cudaError_t launch_restrict_t<float>(hdg_handle *, const float *, float *);
template cudaError_t launch_prolong_add_t<double>(hdg_handle *, const double *, double *);
template cudaError_t launch_prolong_add_t<float>(hdg_handle *, const float *, float *);

cudaError_t launch_to_internal(hdg_handle *h, const double *ext, double *in) {
    size_t n = size_t(h->NF) * h->pp;
    to_internal_kernel<<<blocks(n, 256), 256, 0, h->stream>>>(h->NF, h->pp, ext, in);
    return cudaGetLastError();
}
cudaError_t launch_to_external(hdg_handle *h, const double *in, double *ext) {
    size_t n = size_t(h->NF) * h->pp;
    to_external_kernel<<<blocks(n, 256), 256, 0, h->stream>>>(h->NF, h->pp, in, ext);
    return cudaGetLastError();
}

cudaError_t launch_rhs(hdg_handle *h, const double *r_u, const double *r_h, double *g, double *ycell) {
    size_t n = size_t(h->N) * h->m;
    HDG_DISPATCH_P(h->p, (rhs_cell_kernel<P><<<blocks(n, 256), 256, 0, h->stream>>>(h->N, h->d_W, r_u, r_h, ycell)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    HDG_DISPATCH_P(h->p, (rhs_gather_kernel<P><<<blocks(h->NF, 256), 256, 0, h->stream>>>(h->N, h->NF, ycell, h->d_facet_cell, h->d_facet_edge, h->d_flip, g)));
    return cudaGetLastError();
}

cudaError_t launch_recover(hdg_handle *h, const double *r_u, const double *r_h, const double *lam, double *u,
                           double *hout) {
    size_t n = size_t(h->N) * h->nK;
    HDG_DISPATCH_P(h->p, (recover_kernel<P><<<blocks(n, 256), 256, 0, h->stream>>>(h->N, h->NF, h->d_Rm, h->d_Xb, r_u, r_h, lam, h->d_facet_of, h->d_flip, u, hout)));
    return cudaGetLastError();
}

}  // namespace hdg
