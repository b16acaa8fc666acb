// Geometric V-cycle on the nested P1 levels for the coarse problem of the
// two-level method (Eq. coarse_problem_upwind): damped Jacobi smoothing with
// CSR operators, restriction by the transpose of the midpoint prolongation,
// and a dense inverse on the coarsest level.
#include "common.h"

namespace hdg {

namespace {

inline unsigned blocks(size_t n, int bs) { return unsigned((n + bs - 1) / bs); }

// x_out = x + omega D^-1 (b - A x); first sweep (x = 0): x_out = omega D^-1 b
template <typename T>
__global__ void jacobi_kernel(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                              const T *__restrict__ A, const T *__restrict__ dinv, const T *__restrict__ b,
                              const T *__restrict__ x, T *__restrict__ xout, T omega, int first) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (first) {
        xout[i] = omega * dinv[i] * b[i];
        return;
    }
    T ax = T(0);
    for (int k = rp[i]; k < rp[i + 1]; ++k) ax = fma(A[k], x[col[k]], ax);
    xout[i] = fma(omega * dinv[i], b[i] - ax, x[i]);
}

template <typename T>
__global__ void residual_kernel(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                const T *__restrict__ A, const T *__restrict__ b, const T *__restrict__ x,
                                T *__restrict__ r) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T ax = T(0);
    for (int k = rp[i]; k < rp[i + 1]; ++k) ax = fma(A[k], x[col[k]], ax);
    r[i] = b[i] - ax;
}

template <typename T>
__global__ void restrict_kernel(int nc, const int32_t *__restrict__ cp, const int32_t *__restrict__ ci,
                                const double *__restrict__ cw, const T *__restrict__ rf, T *__restrict__ bc) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    T acc = T(0);
    for (int k = cp[c]; k < cp[c + 1]; ++k) acc = fma(T(cw[k]), rf[ci[k]], acc);
    bc[c] = acc;
}

template <typename T>
__global__ void prolong_add_kernel(int nf, const int32_t *__restrict__ parent, const T *__restrict__ ec,
                                   T *__restrict__ xf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    const int a = parent[2 * i], b = parent[2 * i + 1];
    xf[i] += (a == b) ? ec[a] : T(0.5) * (ec[a] + ec[b]);
}

// x = inv b, one warp per row (inv row-major, n <= 1024)
template <typename T>
__global__ void dense_apply_kernel(const T *__restrict__ inv, int n, const T *__restrict__ b, T *__restrict__ x) {
    const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x % 32;
    if (row >= n) return;
    double acc = 0.0;
    for (int c = lane; c < n; c += 32) acc += double(inv[size_t(row) * n + c]) * double(b[c]);
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) x[row] = T(acc);
}

}  // namespace

template <typename T>
cudaError_t launch_p1_jacobi(const DevLevel &L, const T *A, const T *dinv, const T *b, const T *x, T *xout, T omega,
                             bool first, cudaStream_t s) {
    jacobi_kernel<T><<<blocks(L.nv, 256), 256, 0, s>>>(L.nv, L.row_ptr, L.col, A, dinv, b, x, xout, omega, first ? 1 : 0);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_p1_residual(const DevLevel &L, const T *A, const T *b, const T *x, T *r, cudaStream_t s) {
    residual_kernel<T><<<blocks(L.nv, 256), 256, 0, s>>>(L.nv, L.row_ptr, L.col, A, b, x, r);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_p1_restrict(const DevLevel &coarse, const T *rf, T *bc, cudaStream_t s) {
    restrict_kernel<T><<<blocks(coarse.nv, 256), 256, 0, s>>>(coarse.nv, coarse.child_ptr, coarse.child_idx,
                                                              coarse.child_w, rf, bc);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_p1_prolong_add(const DevLevel &coarse, int nv_fine, const T *ec, T *xf, cudaStream_t s) {
    prolong_add_kernel<T><<<blocks(nv_fine, 256), 256, 0, s>>>(nv_fine, coarse.parent, ec, xf);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_dense_apply(const T *inv, int n, const T *b, T *x, cudaStream_t s) {
    dense_apply_kernel<T><<<blocks(size_t(n) * 32, 256), 256, 0, s>>>(inv, n, b, x);
    return cudaGetLastError();
}

#define HDG_P1_INST(T)                                                                                         \
    template cudaError_t launch_p1_jacobi<T>(const DevLevel &, const T *, const T *, const T *, const T *, T *, \
                                             T, bool, cudaStream_t);                                           \
    template cudaError_t launch_p1_residual<T>(const DevLevel &, const T *, const T *, const T *, T *,           \
                                               cudaStream_t);                                                  \
    template cudaError_t launch_p1_restrict<T>(const DevLevel &, const T *, T *, cudaStream_t);                 \
    template cudaError_t launch_p1_prolong_add<T>(const DevLevel &, int, const T *, T *, cudaStream_t);         \
    template cudaError_t launch_dense_apply<T>(const T *, int, const T *, T *, cudaStream_t);
HDG_P1_INST(double)
HDG_P1_INST(float)

}  // namespace hdg
