// Kernels of the FGMRES driver: deterministic multi-dot products (fixed-order
// block and tree reductions, accumulated in double), multi-AXPY updates for
// classical Gram-Schmidt with re-orthogonalisation, and the tiny serial
// steps (Hessenberg column, Givens rotation, triangular solve) kept on the
// device so the host reads back one residual estimate per iteration.
#include "common.h"

#include <cmath>

namespace hdg {

namespace {

inline unsigned blocks(size_t n, int bs) { return unsigned((n + bs - 1) / bs); }

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[32];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    const int nw = blockDim.x / 32;
    v = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
    if (warp == 0)
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// partial[i][c] = sum over chunk c of V_i . w
template <typename T>
__global__ void __launch_bounds__(256) multidot_kernel(const T *__restrict__ V, size_t ld, const T *__restrict__ w,
                                                       size_t n, double *__restrict__ partial, int nchunk) {
    const int i = blockIdx.y, c = blockIdx.x;
    const size_t len = (n + nchunk - 1) / nchunk;
    const size_t beg = size_t(c) * len, end = beg + len < n ? beg + len : n;
    const T *v = V + size_t(i) * ld;
    double acc = 0.0;
    for (size_t k = beg + threadIdx.x; k < end; k += blockDim.x) acc = fma(double(v[k]), double(w[k]), acc);
    acc = block_sum(acc);
    if (threadIdx.x == 0) partial[size_t(i) * nchunk + c] = acc;
}

__global__ void reduce_partials_kernel(const double *__restrict__ partial, int nchunk, double *__restrict__ out) {
    const int i = blockIdx.x;
    double acc = 0.0;
    for (int c = threadIdx.x; c < nchunk; c += blockDim.x) acc += partial[size_t(i) * nchunk + c];
    acc = block_sum(acc);
    if (threadIdx.x == 0) out[i] = acc;
}

// w += sign * sum_i coef[i] V_i
template <typename T>
__global__ void __launch_bounds__(256) multi_axpy_kernel(T *__restrict__ w, const T *__restrict__ V, size_t ld, int k,
                                                         const double *__restrict__ coef, double sign, size_t n) {
    const size_t idx = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    double acc = 0.0;
    for (int i = 0; i < k; ++i) acc = fma(coef[i], double(V[size_t(i) * ld + idx]), acc);
    w[idx] = T(double(w[idx]) + sign * acc);
}

template <typename T>
__global__ void scale_copy_kernel(const T *__restrict__ w, T *__restrict__ v, const double *__restrict__ denom,
                                  size_t n) {
    const size_t idx = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    v[idx] = T(double(w[idx]) / denom[0]);
}

// Hessenberg column j from the two Gram-Schmidt passes; h[j+1] = ||w||
__global__ void arnoldi_finish_kernel(double *Hcol, const double *h1, const double *h2, const double *nrm2, int j) {
    for (int i = 0; i <= j; ++i) Hcol[i] = h1[i] + h2[i];
    Hcol[j + 1] = sqrt(nrm2[0]);
}

// Apply the previous rotations to column j, form rotation j, update the RHS of
// the least-squares problem; est = |s_{j+1}| / ||b||.  flags: 2 = breakdown,
// 4 = NaN/Inf.
__global__ void givens_kernel(double *Hm, int ldh, double *cs, double *sn, double *sv, int j, const double *bnorm_p,
                              double *est, int32_t *flags) {
    const double bnorm = bnorm_p[0];
    double *col = Hm + size_t(j) * ldh;
    for (int i = 0; i < j; ++i) {
        const double t = cs[i] * col[i] + sn[i] * col[i + 1];
        col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
        col[i] = t;
    }
    const double a = col[j], b = col[j + 1];
    const double den = hypot(a, b);
    int32_t fl = 0;
    if (!(den > 0.0)) {
        cs[j] = 1.0; sn[j] = 0.0;
        fl |= 2;
    } else {
        cs[j] = a / den; sn[j] = b / den;
    }
    if (!(fabs(b) > 1e-300 * (fabs(a) + 1e-300))) fl |= 2;
    col[j] = (den > 0.0) ? den : a;
    col[j + 1] = 0.0;
    sv[j + 1] = -sn[j] * sv[j];
    sv[j] = cs[j] * sv[j];
    est[0] = fabs(sv[j + 1]) / bnorm;
    if (!isfinite(est[0]) || !isfinite(den)) fl |= 4;
    flags[0] = fl;
}

__global__ void hessenberg_solve_kernel(const double *Hm, int ldh, const double *sv, int k, double *y) {
    for (int i = k - 1; i >= 0; --i) {
        double s = sv[i];
        for (int l = i + 1; l < k; ++l) s -= Hm[size_t(l) * ldh + i] * y[l];
        y[i] = s / Hm[size_t(i) * ldh + i];
    }
}

template <typename T>
__global__ void fill_kernel(T *x, T v, size_t n) {
    const size_t idx = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx < n) x[idx] = v;
}

// x += scale * d (refinement correction, FP32 -> FP64)
__global__ void axpby_mixed_kernel(double *x, const float *d, const double *scale, size_t n) {
    const size_t idx = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx < n) x[idx] = fma(scale[0], double(d[idx]), x[idx]);
}

// y = float(x / scale[0])
__global__ void d2f_scaled_kernel(const double *x, float *y, const double *scale, size_t n) {
    const size_t idx = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx < n) y[idx] = float(x[idx] / scale[0]);
}

}  // namespace

template <typename T>
cudaError_t launch_multidot(const T *V, size_t ld, int k, const T *w, size_t n, double *partial, int nchunk,
                            cudaStream_t s) {
    dim3 grid(nchunk, k);
    multidot_kernel<T><<<grid, 256, 0, s>>>(V, ld, w, n, partial, nchunk);
    return cudaGetLastError();
}
cudaError_t launch_reduce_partials(const double *partial, int k, int nchunk, double *out, cudaStream_t s) {
    reduce_partials_kernel<<<k, 256, 0, s>>>(partial, nchunk, out);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_multi_axpy(T *w, const T *V, size_t ld, int k, const double *coef, double sign, size_t n,
                              cudaStream_t s) {
    multi_axpy_kernel<T><<<blocks(n, 256), 256, 0, s>>>(w, V, ld, k, coef, sign, n);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_scale_copy(const T *w, T *v, const double *denom, size_t n, cudaStream_t s) {
    scale_copy_kernel<T><<<blocks(n, 256), 256, 0, s>>>(w, v, denom, n);
    return cudaGetLastError();
}
cudaError_t launch_arnoldi_finish(double *Hcol, const double *h1, const double *h2, const double *nrm2, int j,
                                  cudaStream_t s) {
    arnoldi_finish_kernel<<<1, 1, 0, s>>>(Hcol, h1, h2, nrm2, j);
    return cudaGetLastError();
}
cudaError_t launch_givens(double *Hm, int ldh, double *cs, double *sn, double *sv, int j, const double *bnorm, double *est,
                          int32_t *flags, cudaStream_t s) {
    givens_kernel<<<1, 1, 0, s>>>(Hm, ldh, cs, sn, sv, j, bnorm, est, flags);
    return cudaGetLastError();
}
cudaError_t launch_hessenberg_solve(const double *Hm, int ldh, const double *sv, int k, double *y, cudaStream_t s) {
    hessenberg_solve_kernel<<<1, 1, 0, s>>>(Hm, ldh, sv, k, y);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_fill(T *x, T v, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    fill_kernel<T><<<blocks(n, 256), 256, 0, s>>>(x, v, n);
    return cudaGetLastError();
}
cudaError_t launch_axpby_mixed(double *x, const float *d, const double *scale, size_t n, cudaStream_t s) {
    axpby_mixed_kernel<<<blocks(n, 256), 256, 0, s>>>(x, d, scale, n);
    return cudaGetLastError();
}
cudaError_t launch_d2f_scaled(const double *x, float *y, const double *scale, size_t n, cudaStream_t s) {
    d2f_scaled_kernel<<<blocks(n, 256), 256, 0, s>>>(x, y, scale, n);
    return cudaGetLastError();
}

#define HDG_KRYLOV_INST(T)                                                                                      \
    template cudaError_t launch_multidot<T>(const T *, size_t, int, const T *, size_t, double *, int,           \
                                            cudaStream_t);                                                      \
    template cudaError_t launch_multi_axpy<T>(T *, const T *, size_t, int, const double *, double, size_t,      \
                                              cudaStream_t);                                                    \
    template cudaError_t launch_scale_copy<T>(const T *, T *, const double *, size_t, cudaStream_t);            \
    template cudaError_t launch_fill<T>(T *, T, size_t, cudaStream_t);
HDG_KRYLOV_INST(double)
HDG_KRYLOV_INST(float)

}  // namespace hdg
