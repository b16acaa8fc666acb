// Kernels of the FGMRES driver: deterministic multi-dot products (fixed-order
// block and tree reductions, accumulated in double), multi-AXPY updates for
// classical Gram-Schmidt with re-orthogonalisation, and the tiny serial
// steps (Hessenberg column, Givens rotation, triangular solve) kept on the
// device so the host reads back one residual estimate per iteration.
#include "common.h"

#include <cmath>

namespace hdg {

// launch family of this file for pdl_launch (Krylov and copy kernels)
constexpr unsigned kPdlFamily = 4;

namespace {

inline unsigned blocks(size_t n, int bs) { return unsigned((n + bs - 1) / bs); }

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[32];
    __syncthreads();      // red[] may still be read by a previous call
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
    T acc = T(0);
    for (size_t k = beg + threadIdx.x; k < end; k += blockDim.x) acc = fma(v[k], w[k], acc);
    const double tot = block_sum(double(acc));
    if (threadIdx.x == 0) partial[size_t(i) * nchunk + c] = tot;
}

// v . w in one launch: block c sums chunk c (as multidot_kernel), the last
// block to finish adds the nchunk partials (as reduce_partials_kernel: the
// same order, the same result) into out[0], optionally its square root into
// root_a / root_b and a hand-over to the host (pub, seq)
template <typename T>
__device__ __forceinline__ void dot1_kernel_impl(int bid_, int nb_, const T *__restrict__ v, const T *__restrict__ w,
                                                 size_t n, double *__restrict__ partial, int nchunk,
                                                 unsigned int *__restrict__ counter, double *__restrict__ out,
                                                 HostValue *pub, int32_t seq, double *root_a, double *root_b) {
    __shared__ bool last;
    const int c = bid_;
    const size_t len = (n + nchunk - 1) / nchunk;
    const size_t beg = size_t(c) * len, end = beg + len < n ? beg + len : n;
    T acc = T(0);
    for (size_t k = beg + threadIdx.x; k < end; k += blockDim.x) acc = fma(v[k], w[k], acc);
    const double tot = block_sum(double(acc));
    if (threadIdx.x == 0) {
        partial[c] = tot;
        __threadfence();                       // the partial is visible before the count
        last = atomicAdd(counter, 1u) == nb_ - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double a = 0.0;
    for (int i = threadIdx.x; i < nchunk; i += blockDim.x) a += partial[i];
    a = block_sum(a);
    if (threadIdx.x == 0) {
        *counter = 0u;
        out[0] = a;
        if (root_a || root_b) {
            const double r = sqrt(a);
            if (root_a) *root_a = r;
            if (root_b) *root_b = r;
        }
        if (pub) {
            pub->v = a;
            __threadfence_system();
            *reinterpret_cast<volatile int32_t *>(&pub->seq) = seq;
        }
    }
}
template <typename T>
__global__ void __launch_bounds__(256) dot1_kernel(const T *__restrict__ v, const T *__restrict__ w, size_t n,
                                                   double *__restrict__ partial, int nchunk,
                                                   unsigned int *__restrict__ counter, double *__restrict__ out,
                                                   HostValue *pub, int32_t seq, double *root_a, double *root_b) {
    pdl_wait();
    dot1_kernel_impl<T>(blockIdx.x, gridDim.x, v, w, n, partial, nchunk, counter, out, pub, seq, root_a, root_b);
}
template <typename T>
struct dot1_kernel_args {
    int nb_;
    const T *v;
    const T *w;
    size_t n;
    double *partial;
    int nchunk;
    unsigned int *counter;
    double *out;
    HostValue *pub;
    int32_t seq;
    double *root_a;
    double *root_b;
};
template <typename T>
__global__ void __launch_bounds__(256) dot1_kernel_multi(const __grid_constant__ MultiP<dot1_kernel_args<T>> M) {
    pdl_wait();
    int b_;
    const dot1_kernel_args<T> &q_ = M.a[merge_find(M.start, M.n, b_)];
    dot1_kernel_impl<T>(b_, q_.nb_, q_.v, q_.w, q_.n, q_.partial, q_.nchunk, q_.counter, q_.out, q_.pub, q_.seq,
        q_.root_a, q_.root_b);
}
template <typename T>
void dot1_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, const T *v, const T *w, size_t n,
                    double *partial, int nchunk, unsigned int *counter, double *out, HostValue *pub, int32_t seq,
                    double *root_a, double *root_b) {
    if (Recorder *r_ = batch_recorder()) {
        dot1_kernel_args<T> q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.v = v;
        q_.w = w;
        q_.n = n;
        q_.partial = partial;
        q_.nchunk = nchunk;
        q_.counter = counter;
        q_.out = out;
        q_.pub = pub;
        q_.seq = seq;
        q_.root_a = root_a;
        q_.root_b = root_b;
        batch_record(r_, reinterpret_cast<const void *>(&dot1_kernel_multi<T>), q_, grid_, block_, smem_, kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &dot1_kernel<T>, grid_, block_, smem_, s_, v, w, n, partial, nchunk, counter, out, pub, seq, root_a, root_b);
}


// out[i] = sum of the partials of vector i; with pub, block 0 also hands its
// sum to the host (page-locked HostValue: the value, a system fence, seq);
// root_a / root_b (may be null) receive the square root of block 0's sum
__global__ void reduce_partials_kernel(const double *__restrict__ partial, int nchunk, double *__restrict__ out,
                                       HostValue *pub, int32_t seq, double *root_a, double *root_b) {
    const int i = blockIdx.x;
    double acc = 0.0;
    for (int c = threadIdx.x; c < nchunk; c += blockDim.x) acc += partial[size_t(i) * nchunk + c];
    acc = block_sum(acc);
    if (threadIdx.x == 0) {
        out[i] = acc;
        if (i == 0 && (root_a || root_b)) {
            const double r = sqrt(acc);
            if (root_a) *root_a = r;
            if (root_b) *root_b = r;
        }
        if (pub && i == 0) {
            pub->v = acc;
            __threadfence_system();
            *reinterpret_cast<volatile int32_t *>(&pub->seq) = seq;
        }
    }
}

// w += sign * sum_i coef[i] V_i
template <typename T>
__device__ __forceinline__ void multi_axpy_kernel_impl(int bid_, int nb_, T *__restrict__ w, const T *__restrict__ V,
                                                       size_t ld, int k, const double *__restrict__ coef, double sign,
                                                       size_t n) {
    __shared__ T cf[66];
    for (int i = threadIdx.x; i < k; i += blockDim.x) cf[i] = T(sign * coef[i]);
    __syncthreads();
    const size_t idx = size_t(bid_) * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    T acc = w[idx];
    for (int i = 0; i < k; ++i) acc = fma(cf[i], V[size_t(i) * ld + idx], acc);
    w[idx] = acc;
}
template <typename T>
__global__ void __launch_bounds__(256) multi_axpy_kernel(T *__restrict__ w, const T *__restrict__ V, size_t ld, int k,
                                                         const double *__restrict__ coef, double sign, size_t n) {
    pdl_wait();
    multi_axpy_kernel_impl<T>(blockIdx.x, gridDim.x, w, V, ld, k, coef, sign, n);
}
template <typename T>
struct multi_axpy_kernel_args {
    int nb_;
    T *w;
    const T *V;
    size_t ld;
    int k;
    const double *coef;
    double sign;
    size_t n;
};
template <typename T>
__global__ void __launch_bounds__(256) multi_axpy_kernel_multi(const __grid_constant__ MultiP<multi_axpy_kernel_args<T>> M) {
    pdl_wait();
    int b_;
    const multi_axpy_kernel_args<T> &q_ = M.a[merge_find(M.start, M.n, b_)];
    multi_axpy_kernel_impl<T>(b_, q_.nb_, q_.w, q_.V, q_.ld, q_.k, q_.coef, q_.sign, q_.n);
}
template <typename T>
void multi_axpy_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, T *w, const T *V, size_t ld,
                          int k, const double *coef, double sign, size_t n) {
    if (Recorder *r_ = batch_recorder()) {
        multi_axpy_kernel_args<T> q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.w = w;
        q_.V = V;
        q_.ld = ld;
        q_.k = k;
        q_.coef = coef;
        q_.sign = sign;
        q_.n = n;
        batch_record(r_, reinterpret_cast<const void *>(&multi_axpy_kernel_multi<T>), q_, grid_, block_, smem_, kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &multi_axpy_kernel<T>, grid_, block_, smem_, s_, w, V, ld, k, coef, sign, n);
}


// 1 / d[0] in FP64, formed once per block (FP64 division is slow on this part;
// every thread reaches the barrier, so call it before any early return)
__device__ __forceinline__ double block_recip(const double *d) {
    __shared__ double r;
    if (threadIdx.x == 0) r = 1.0 / d[0];
    __syncthreads();
    return r;
}

// FP64 FGMRES with the FP32 preconditioner: v = w / h (h from the Givens step
// of the previous Arnoldi step, reciprocal once per block) stored as the next
// FP64 basis vector, and rounded to FP32 as the preconditioner's input; with
// hnext null, w is the basis vector itself and is only rounded.
__global__ void scale_round_kernel(const double *__restrict__ w, const double *__restrict__ hnext,
                                   double *__restrict__ v64, float *__restrict__ v32, size_t n) {
    __shared__ double inv_h;
    if (hnext != nullptr) {
        if (threadIdx.x == 0) inv_h = 1.0 / hnext[0];
        __syncthreads();
    }
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = w[i];
    if (hnext != nullptr) {
        v = v * inv_h;
        v64[i] = v;
    }
    v32[i] = float(v);
}

// the FP32 preconditioner's output widened to the FP64 basis Z
__global__ void widen_kernel(const float *__restrict__ a, double *__restrict__ b, size_t n) {
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) b[i] = double(a[i]);
}

template <typename T>
__device__ __forceinline__ void scale_copy_kernel_impl(int bid_, int nb_, const T *__restrict__ w, T *__restrict__ v,
                                                       const double *__restrict__ denom, size_t n) {
    const double inv = block_recip(denom);
    const size_t idx = size_t(bid_) * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    v[idx] = w[idx] * T(inv);
}
template <typename T>
__global__ void scale_copy_kernel(const T *__restrict__ w, T *__restrict__ v, const double *__restrict__ denom,
                                  size_t n) {
    pdl_wait();
    scale_copy_kernel_impl<T>(blockIdx.x, gridDim.x, w, v, denom, n);
}
template <typename T>
struct scale_copy_kernel_args {
    int nb_;
    const T *w;
    T *v;
    const double *denom;
    size_t n;
};
template <typename T>
__global__ void scale_copy_kernel_multi(const __grid_constant__ MultiP<scale_copy_kernel_args<T>> M) {
    pdl_wait();
    int b_;
    const scale_copy_kernel_args<T> &q_ = M.a[merge_find(M.start, M.n, b_)];
    scale_copy_kernel_impl<T>(b_, q_.nb_, q_.w, q_.v, q_.denom, q_.n);
}
template <typename T>
void scale_copy_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, const T *w, T *v,
                          const double *denom, size_t n) {
    if (Recorder *r_ = batch_recorder()) {
        scale_copy_kernel_args<T> q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.w = w;
        q_.v = v;
        q_.denom = denom;
        q_.n = n;
        batch_record(r_, reinterpret_cast<const void *>(&scale_copy_kernel_multi<T>), q_, grid_, block_, smem_, kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &scale_copy_kernel<T>, grid_, block_, smem_, s_, w, v, denom, n);
}


// y = R^-1 s for the leading k x k upper triangle R of the rotated Hessenberg
// matrix (column-major, leading dimension ldh): the triangle and s are first
// loaded into shared memory by the whole block, then one thread substitutes
// backwards (k <= 64)
__device__ __forceinline__ void hessenberg_solve_kernel_impl(int bid_, int nb_, const double *Hm, int ldh,
                                                             const double *sv, int k, double *y) {
    __shared__ double R[64][65], sS[64], yS[64];
    for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
        const int l = t / k, i = t % k;            // column l, row i
        if (i <= l) R[i][l] = Hm[size_t(l) * ldh + i];
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) sS[i] = sv[i];
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int i = k - 1; i >= 0; --i) {
        double s = sS[i];
        for (int l = i + 1; l < k; ++l) s -= R[i][l] * yS[l];
        yS[i] = s / R[i][i];
        y[i] = yS[i];
    }
}
__global__ void hessenberg_solve_kernel(const double *Hm, int ldh, const double *sv, int k, double *y) {
    pdl_wait();
    hessenberg_solve_kernel_impl(blockIdx.x, gridDim.x, Hm, ldh, sv, k, y);
}
struct hessenberg_solve_kernel_args {
    int nb_;
    const double *Hm;
    int ldh;
    const double *sv;
    int k;
    double *y;
};
__global__ void hessenberg_solve_kernel_multi(const __grid_constant__ MultiP<hessenberg_solve_kernel_args> M) {
    pdl_wait();
    int b_;
    const hessenberg_solve_kernel_args &q_ = M.a[merge_find(M.start, M.n, b_)];
    hessenberg_solve_kernel_impl(b_, q_.nb_, q_.Hm, q_.ldh, q_.sv, q_.k, q_.y);
}
void hessenberg_solve_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, const double *Hm,
                                int ldh, const double *sv, int k, double *y) {
    if (Recorder *r_ = batch_recorder()) {
        hessenberg_solve_kernel_args q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.Hm = Hm;
        q_.ldh = ldh;
        q_.sv = sv;
        q_.k = k;
        q_.y = y;
        batch_record(r_, reinterpret_cast<const void *>(&hessenberg_solve_kernel_multi), q_, grid_, block_, smem_, kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &hessenberg_solve_kernel, grid_, block_, smem_, s_, Hm, ldh, sv, k, y);
}


template <typename T>
__device__ __forceinline__ void fill_kernel_impl(int bid_, int nb_, T *x, T v, size_t n) {
    const size_t idx = size_t(bid_) * blockDim.x + threadIdx.x;
    if (idx < n) x[idx] = v;
}
template <typename T>
__global__ void fill_kernel(T *x, T v, size_t n) {
    pdl_wait();
    fill_kernel_impl<T>(blockIdx.x, gridDim.x, x, v, n);
}
template <typename T>
struct fill_kernel_args {
    int nb_;
    T *x;
    T v;
    size_t n;
};
template <typename T>
__global__ void fill_kernel_multi(const __grid_constant__ MultiP<fill_kernel_args<T>> M) {
    pdl_wait();
    int b_;
    const fill_kernel_args<T> &q_ = M.a[merge_find(M.start, M.n, b_)];
    fill_kernel_impl<T>(b_, q_.nb_, q_.x, q_.v, q_.n);
}
template <typename T>
void fill_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, T *x, T v, size_t n) {
    if (Recorder *r_ = batch_recorder()) {
        fill_kernel_args<T> q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.x = x;
        q_.v = v;
        q_.n = n;
        batch_record(r_, reinterpret_cast<const void *>(&fill_kernel_multi<T>), q_, grid_, block_, smem_, kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &fill_kernel<T>, grid_, block_, smem_, s_, x, v, n);
}


// y = float(x / scale[0])
// b = float(x / scale[0]) and z = 0 on n entries, with ||b||^2 (float sums per
// thread over a grid-stride range, block sums in double, the last block adding
// the block sums in block order) into out[0] and its square root into root_a
// and root_b: an inner solve's right-hand side, its zero initial guess and
// the norm that starts it, in one pass
__device__ __forceinline__ void d2f_norm_kernel_impl(int bid_, int nb_, const double *__restrict__ x,
                                                     float *__restrict__ y, float *__restrict__ z,
                                                     const double *scale, size_t n, double *partial,
                                                     unsigned int *counter, double *out, double *root_a,
                                                     double *root_b) {
    __shared__ bool last;
    // kU loads in flight per thread before their results are used (the grid
    // is a few blocks per SM), the first kU issued before the block waits for
    // the reciprocal; each thread still adds its entries in index order
    constexpr int kU = 8;
    const size_t stride = size_t(nb_) * blockDim.x, i0 = size_t(bid_) * blockDim.x + threadIdx.x;
    double a[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) a[u] = i0 + u * stride < n ? x[i0 + u * stride] : 0.0;
    const double inv = block_recip(scale);
    float acc = 0.0f;
    for (size_t i = i0; i < n; i += kU * stride) {
        if (i != i0) {
#pragma unroll
            for (int u = 0; u < kU; ++u) a[u] = i + u * stride < n ? x[i + u * stride] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            if (i + u * stride < n) {
                const float v = float(a[u] * inv);
                y[i + u * stride] = v;
                z[i + u * stride] = 0.0f;
                acc = fmaf(v, v, acc);
            }
        }
    }
    const double tot = block_sum(double(acc));
    if (threadIdx.x == 0) {
        partial[bid_] = tot;
        __threadfence();                       // the partial is visible before the count
        last = atomicAdd(counter, 1u) == unsigned(nb_) - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double t = 0.0;
    for (int i = threadIdx.x; i < nb_; i += blockDim.x) t += partial[i];
    t = block_sum(t);
    if (threadIdx.x == 0) {
        *counter = 0u;
        out[0] = t;
        const double r = sqrt(t);
        if (root_a) *root_a = r;
        if (root_b) *root_b = r;
    }
}
__global__ void __launch_bounds__(256) d2f_norm_kernel(const double *x, float *y, float *z, const double *scale,
                                                       size_t n, double *partial, unsigned int *counter, double *out,
                                                       double *root_a, double *root_b) {
    pdl_wait();
    d2f_norm_kernel_impl(blockIdx.x, gridDim.x, x, y, z, scale, n, partial, counter, out, root_a, root_b);
}
struct d2f_norm_kernel_args {
    int nb_;
    const double *x;
    float *y;
    float *z;
    const double *scale;
    size_t n;
    double *partial;
    unsigned int *counter;
    double *out;
    double *root_a;
    double *root_b;
};
__global__ void __launch_bounds__(256) d2f_norm_kernel_multi(const __grid_constant__ MultiP<d2f_norm_kernel_args> M) {
    pdl_wait();
    int b_;
    const d2f_norm_kernel_args &q_ = M.a[merge_find(M.start, M.n, b_)];
    d2f_norm_kernel_impl(b_, q_.nb_, q_.x, q_.y, q_.z, q_.scale, q_.n, q_.partial, q_.counter, q_.out, q_.root_a,
                         q_.root_b);
}
void d2f_norm_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, const double *x, float *y,
                        float *z, const double *scale, size_t n, double *partial, unsigned int *counter, double *out,
                        double *root_a, double *root_b) {
    if (Recorder *r_ = batch_recorder()) {
        d2f_norm_kernel_args q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.x = x;
        q_.y = y;
        q_.z = z;
        q_.scale = scale;
        q_.n = n;
        q_.partial = partial;
        q_.counter = counter;
        q_.out = out;
        q_.root_a = root_a;
        q_.root_b = root_b;
        batch_record(r_, reinterpret_cast<const void *>(&d2f_norm_kernel_multi), q_, grid_, block_, smem_, kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &d2f_norm_kernel, grid_, block_, smem_, s_, x, y, z, scale, n, partial, counter, out, root_a,
               root_b);
}

__device__ __forceinline__ void d2f_scaled_kernel_impl(int bid_, int nb_, const double *x, float *y,
                                                       const double *scale, size_t n) {
    const double inv = block_recip(scale);
    const size_t idx = size_t(bid_) * blockDim.x + threadIdx.x;
    if (idx < n) y[idx] = float(x[idx] * inv);
}
__global__ void d2f_scaled_kernel(const double *x, float *y, const double *scale, size_t n) {
    pdl_wait();
    d2f_scaled_kernel_impl(blockIdx.x, gridDim.x, x, y, scale, n);
}
struct d2f_scaled_kernel_args {
    int nb_;
    const double *x;
    float *y;
    const double *scale;
    size_t n;
};
__global__ void d2f_scaled_kernel_multi(const __grid_constant__ MultiP<d2f_scaled_kernel_args> M) {
    pdl_wait();
    int b_;
    const d2f_scaled_kernel_args &q_ = M.a[merge_find(M.start, M.n, b_)];
    d2f_scaled_kernel_impl(b_, q_.nb_, q_.x, q_.y, q_.scale, q_.n);
}
void d2f_scaled_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, const double *x, float *y,
                          const double *scale, size_t n) {
    if (Recorder *r_ = batch_recorder()) {
        d2f_scaled_kernel_args q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.x = x;
        q_.y = y;
        q_.scale = scale;
        q_.n = n;
        batch_record(r_, reinterpret_cast<const void *>(&d2f_scaled_kernel_multi), q_, grid_, block_, smem_, kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &d2f_scaled_kernel, grid_, block_, smem_, s_, x, y, scale, n);
}



// ---------------------------------------------------------------- fused CGS2
// Vectors of the Krylov basis are padded to a multiple of 16 bytes (zero
// padding) so every thread moves 16-byte words.  Arithmetic stays in the
// vector precision per element (GB300's FP64 and conversion throughput is a
// small fraction of its FP32 throughput); only the per-block partial sums are
// combined in double.
template <typename T> struct V16;
template <> struct V16<float> {
    using type = float4;
    using acc = float;
    __device__ static float dot(const float4 a, const float4 b) {
        return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
    }
    __device__ static float4 axpy(float c, const float4 v, const float4 w) {
        return make_float4(fmaf(c, v.x, w.x), fmaf(c, v.y, w.y), fmaf(c, v.z, w.z), fmaf(c, v.w, w.w));
    }
    __device__ static float4 scale(const float4 v, float s) { return make_float4(v.x * s, v.y * s, v.z * s, v.w * s); }
};
template <> struct V16<double> {
    using type = double2;
    using acc = double;
    __device__ static double dot(const double2 a, const double2 b) { return fma(a.x, b.x, a.y * b.y); }
    __device__ static double2 axpy(double c, const double2 v, const double2 w) {
        return make_double2(fma(c, v.x, w.x), fma(c, v.y, w.y));
    }
    __device__ static double2 scale(const double2 v, double s) { return make_double2(v.x * s, v.y * s); }
};

// Partial sums of V_i . w for i < k over this block's grid-stride range, in
// groups of kGroup vectors (one pass over w per group, kGroup accumulators per
// thread), then the last block to finish adds the partials in a fixed order
// (finish_partials: deterministic).
constexpr int kGroup = 16;

template <typename T>
__device__ void dots_and_finish(const typename V16<T>::type *__restrict__ V, size_t ld4, int k,
                                const typename V16<T>::type *w, size_t n4, double *partial,
                                unsigned int *counter, double *out, bool *is_last) {
    using A = typename V16<T>::acc;
    __shared__ bool last;
    __shared__ A red[kGroup][9];
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nwarp = blockDim.x / 32;
    for (int i0 = 0; i0 < k; i0 += kGroup) {
        A acc[kGroup];
#pragma unroll
        for (int g = 0; g < kGroup; ++g) acc[g] = A(0);
        for (size_t idx = size_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < n4; idx += size_t(gridDim.x) * blockDim.x) {
            const typename V16<T>::type wv = w[idx];
#pragma unroll
            for (int g = 0; g < kGroup; ++g)
                if (i0 + g < k) acc[g] += V16<T>::dot(V[size_t(i0 + g) * ld4 + idx], wv);
        }
#pragma unroll
        for (int g = 0; g < kGroup; ++g) {
            A v = acc[g];
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == 0) red[g][warp] = v;
        }
        __syncthreads();
        if (threadIdx.x < kGroup && i0 + int(threadIdx.x) < k) {
            A v = A(0);
            for (int q = 0; q < nwarp; ++q) v += red[threadIdx.x][q];
            partial[size_t(i0 + threadIdx.x) * gridDim.x + blockIdx.x] = double(v);
        }
        __syncthreads();
    }
    if (threadIdx.x < kGroup) __threadfence();  // the writers' partials are visible before the count
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    *is_last = last;
    if (!last) return;
    __threadfence();
    finish_partials(partial, int(gridDim.x), k, out);
    if (threadIdx.x == 0) *counter = 0u;
}

// w -= V c over this block's grid-stride range, coefficients staged in shared
// memory in the vector precision
template <typename T>
__device__ void block_update(const typename V16<T>::type *__restrict__ V, size_t ld4, int k,
                             typename V16<T>::type *w, size_t n4, const double *c) {
    __shared__ T cs_[66];
    for (int i = threadIdx.x; i < k; i += blockDim.x) cs_[i] = T(-c[i]);
    __syncthreads();
    for (size_t idx = size_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < n4; idx += size_t(gridDim.x) * blockDim.x) {
        typename V16<T>::type acc = w[idx];
        for (int i = 0; i < k; ++i) acc = V16<T>::axpy(cs_[i], V[size_t(i) * ld4 + idx], acc);
        w[idx] = acc;
    }
    __syncthreads();
}

// w -= V h1, then pass 2: h2 = V^T w
template <typename T>
__global__ void __launch_bounds__(256) gs_update_dots_kernel(const T *V, size_t ld, int k, T *w, size_t n,
                                                             const double *h1, double *partial, unsigned int *counter,
                                                             double *h2) {
    using V4 = typename V16<T>::type;
    const size_t ld4 = ld / (16 / sizeof(T)), n4 = n / (16 / sizeof(T));
    const V4 *V4p = reinterpret_cast<const V4 *>(V);
    V4 *w4 = reinterpret_cast<V4 *>(w);
    block_update<T>(V4p, ld4, k, w4, n4, h1);
    bool last;
    dots_and_finish<T>(V4p, ld4, k, w4, n4, partial, counter, h2, &last);
}

// w -= V h2 (h2 null: w -= V h1, one classical Gram-Schmidt pass) and
// ||w||^2 in the same pass; the last block adds the per-block partials and
// forms Hessenberg column j (h1 + h2, or h1 alone;
// h_{j+1,j} = ||w||), applies the previous Givens rotations, forms rotation j,
// updates the least-squares right-hand side and writes the residual
// estimate |s_{j+1}| / ||b|| and the flags (2: breakdown, 4: NaN/Inf) to rb.
template <typename T>
__device__ __forceinline__ void gs_update_norm_givens_kernel_impl(int bid_, int nb_, const T *V, size_t ld, int k,
                                                                  T *w, size_t n, const double *h1, const double *h2,
                                                                  double *partial, unsigned int *counter,
                                                                  double *nrm2, double *Hm, int ldh, double *cs,
                                                                  double *sn, double *sv, int j, const double *bnorm,
                                                                  ReadBack *rb, ReadBack *host_rb) {
    using V4 = typename V16<T>::type;
    using A = typename V16<T>::acc;
    const size_t ld4 = ld / (16 / sizeof(T)), n4 = n / (16 / sizeof(T));
    const V4 *V4p = reinterpret_cast<const V4 *>(V);
    V4 *w4 = reinterpret_cast<V4 *>(w);
    const double *c = h2 ? h2 : h1;
    __shared__ T cs_[66];
    __shared__ A red[32];
    __shared__ double redd[32];
    __shared__ bool last;
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nwarp = blockDim.x / 32;
    for (int i = threadIdx.x; i < k; i += blockDim.x) cs_[i] = T(-c[i]);
    __syncthreads();
    // the update and ||w||^2 in one pass: each updated value is squared from registers
    A nrm = A(0);
    for (size_t idx = size_t(bid_) * blockDim.x + threadIdx.x; idx < n4; idx += size_t(nb_) * blockDim.x) {
        V4 acc = w4[idx];
        for (int i = 0; i < k; ++i) acc = V16<T>::axpy(cs_[i], V4p[size_t(i) * ld4 + idx], acc);
        w4[idx] = acc;
        nrm += V16<T>::dot(acc, acc);
    }
    for (int off = 16; off > 0; off >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, off);
    if (lane == 0) red[warp] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
        A t = A(0);
        for (int q = 0; q < nwarp; ++q) t += red[q];
        partial[bid_] = double(t);
        __threadfence();                       // the partial is visible before the count
        last = atomicAdd(counter, 1u) == nb_ - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the Hessenberg column and the previous rotations into shared memory (one
    // load per thread, alongside the partials), so that the sequential
    // rotations below touch no global memory
    __shared__ double colS[66], csS[66], snS[66];
    for (int i = threadIdx.x; i <= j; i += blockDim.x) colS[i] = h2 ? h1[i] + h2[i] : h1[i];
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
        csS[i] = cs[i];
        snS[i] = sn[i];
    }
    // the last block adds the partials with all its threads, in a fixed order
    // (thread t: partials t, t + blockDim, ...; then the warp tree; then the warps)
    double v = 0.0;
    for (unsigned b = threadIdx.x; b < nb_; b += blockDim.x) v += partial[b];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) redd[warp] = v;
    __syncthreads();
    if (threadIdx.x != 0) return;
    const double svj = sv[j], bn = bnorm[0];
    double ww = 0.0;
    for (int q = 0; q < nwarp; ++q) ww += redd[q];
    *counter = 0u;
    nrm2[0] = ww;
    colS[j + 1] = sqrt(ww);
    for (int i = 0; i < j; ++i) {
        const double t = csS[i] * colS[i] + snS[i] * colS[i + 1];
        colS[i + 1] = -snS[i] * colS[i] + csS[i] * colS[i + 1];
        colS[i] = t;
    }
    double *col = Hm + size_t(j) * ldh;
    for (int i = 0; i < j; ++i) col[i] = colS[i];
    const double a = colS[j], b = colS[j + 1];
    const double den = hypot(a, b);
    int32_t fl = 0;
    double cj = 1.0, sj = 0.0;
    if (!(den > 0.0)) {
        fl |= 2;
    } else {
        cj = a / den;
        sj = b / den;
    }
    cs[j] = cj;
    sn[j] = sj;
    if (!(fabs(b) > 1e-300 * (fabs(a) + 1e-300))) fl |= 2;
    col[j] = (den > 0.0) ? den : a;
    col[j + 1] = 0.0;
    sv[j + 1] = -sj * svj;
    sv[j] = cj * svj;
    const double est = fabs(-sj * svj) / bn;
    if (!isfinite(est) || !isfinite(den)) fl |= 4;
    rb->est = est;
    rb->flags = fl;
    rb->hnext = b;
    if (host_rb) {
        // the page-locked copy the host polls: the fields, a system-scope fence,
        // then the step number, so that the host may read the fields once it sees it
        host_rb->est = est;
        host_rb->flags = fl;
        host_rb->hnext = b;
        __threadfence_system();
        *reinterpret_cast<volatile int32_t *>(&host_rb->seq) = j + 1;
    }
}
template <typename T>
__global__ void __launch_bounds__(256) gs_update_norm_givens_kernel(const T *V, size_t ld, int k, T *w, size_t n,
                                                                    const double *h1, const double *h2,
                                                                    double *partial, unsigned int *counter,
                                                                    double *nrm2, double *Hm, int ldh, double *cs,
                                                                    double *sn, double *sv, int j,
                                                                    const double *bnorm, ReadBack *rb,
                                                                    ReadBack *host_rb) {
    pdl_wait();
    gs_update_norm_givens_kernel_impl<T>(blockIdx.x, gridDim.x, V, ld, k, w, n, h1, h2, partial, counter, nrm2, Hm,
        ldh, cs, sn, sv, j, bnorm, rb, host_rb);
}
template <typename T>
struct gs_update_norm_givens_kernel_args {
    int nb_;
    const T *V;
    size_t ld;
    int k;
    T *w;
    size_t n;
    const double *h1;
    const double *h2;
    double *partial;
    unsigned int *counter;
    double *nrm2;
    double *Hm;
    int ldh;
    double *cs;
    double *sn;
    double *sv;
    int j;
    const double *bnorm;
    ReadBack *rb;
    ReadBack *host_rb;
};
template <typename T>
__global__ void __launch_bounds__(256) gs_update_norm_givens_kernel_multi(const __grid_constant__ MultiP<gs_update_norm_givens_kernel_args<T>> M) {
    pdl_wait();
    int b_;
    const gs_update_norm_givens_kernel_args<T> &q_ = M.a[merge_find(M.start, M.n, b_)];
    gs_update_norm_givens_kernel_impl<T>(b_, q_.nb_, q_.V, q_.ld, q_.k, q_.w, q_.n, q_.h1, q_.h2, q_.partial,
        q_.counter, q_.nrm2, q_.Hm, q_.ldh, q_.cs, q_.sn, q_.sv, q_.j, q_.bnorm, q_.rb, q_.host_rb);
}
template <typename T>
void gs_update_norm_givens_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, const T *V,
                                     size_t ld, int k, T *w, size_t n, const double *h1, const double *h2,
                                     double *partial, unsigned int *counter, double *nrm2, double *Hm, int ldh,
                                     double *cs, double *sn, double *sv, int j, const double *bnorm, ReadBack *rb,
                                     ReadBack *host_rb) {
    if (Recorder *r_ = batch_recorder()) {
        gs_update_norm_givens_kernel_args<T> q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.V = V;
        q_.ld = ld;
        q_.k = k;
        q_.w = w;
        q_.n = n;
        q_.h1 = h1;
        q_.h2 = h2;
        q_.partial = partial;
        q_.counter = counter;
        q_.nrm2 = nrm2;
        q_.Hm = Hm;
        q_.ldh = ldh;
        q_.cs = cs;
        q_.sn = sn;
        q_.sv = sv;
        q_.j = j;
        q_.bnorm = bnorm;
        q_.rb = rb;
        q_.host_rb = host_rb;
        batch_record(r_, reinterpret_cast<const void *>(&gs_update_norm_givens_kernel_multi<T>), q_, grid_, block_, smem_, kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &gs_update_norm_givens_kernel<T>, grid_, block_, smem_, s_, V, ld, k, w, n, h1, h2, partial, counter, nrm2, Hm,
        ldh, cs, sn, sv, j, bnorm, rb, host_rb);
}


// v_{j+1} = w / h_{j+1,j}  (the unrotated norm kept in rb->hnext)
template <typename T>
__device__ __forceinline__ void gs_scale_kernel_impl(int bid_, int nb_, const T *w, T *v, size_t n,
                                                     const ReadBack *rb) {
    using V4 = typename V16<T>::type;
    const size_t n4 = n / (16 / sizeof(T));
    const T inv = T(block_recip(&rb->hnext));
    const size_t idx = size_t(bid_) * blockDim.x + threadIdx.x;
    if (idx >= n4) return;
    reinterpret_cast<V4 *>(v)[idx] = V16<T>::scale(reinterpret_cast<const V4 *>(w)[idx], inv);
}
template <typename T>
__global__ void gs_scale_kernel(const T *w, T *v, size_t n, const ReadBack *rb) {
    pdl_wait();
    gs_scale_kernel_impl<T>(blockIdx.x, gridDim.x, w, v, n, rb);
}
template <typename T>
struct gs_scale_kernel_args {
    int nb_;
    const T *w;
    T *v;
    size_t n;
    const ReadBack *rb;
};
template <typename T>
__global__ void gs_scale_kernel_multi(const __grid_constant__ MultiP<gs_scale_kernel_args<T>> M) {
    pdl_wait();
    int b_;
    const gs_scale_kernel_args<T> &q_ = M.a[merge_find(M.start, M.n, b_)];
    gs_scale_kernel_impl<T>(b_, q_.nb_, q_.w, q_.v, q_.n, q_.rb);
}
template <typename T>
void gs_scale_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, const T *w, T *v, size_t n,
                        const ReadBack *rb) {
    if (Recorder *r_ = batch_recorder()) {
        gs_scale_kernel_args<T> q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.w = w;
        q_.v = v;
        q_.n = n;
        q_.rb = rb;
        batch_record(r_, reinterpret_cast<const void *>(&gs_scale_kernel_multi<T>), q_, grid_, block_, smem_, kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &gs_scale_kernel<T>, grid_, block_, smem_, s_, w, v, n, rb);
}


}  // namespace

template <typename T>
cudaError_t launch_multidot(const T *V, size_t ld, int k, const T *w, size_t n, double *partial, int nchunk,
                            cudaStream_t s) {
    dim3 grid(nchunk, k);
    multidot_kernel<T><<<grid, 256, 0, s>>>(V, ld, w, n, partial, nchunk);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_dot1(const T *v, const T *w, size_t n, double *partial, int nchunk, unsigned int *counter,
                        double *out, HostValue *pub, int32_t seq, double *root_a, double *root_b, cudaStream_t s) {
    dot1_kernel_go<T>(nchunk, 256, 0, s, v, w, n, partial, nchunk, counter, out, pub, seq, root_a, root_b);
    return cudaGetLastError();
}
template cudaError_t launch_dot1<double>(const double *, const double *, size_t, double *, int, unsigned int *,
                                         double *, HostValue *, int32_t, double *, double *, cudaStream_t);
template cudaError_t launch_dot1<float>(const float *, const float *, size_t, double *, int, unsigned int *, double *,
                                        HostValue *, int32_t, double *, double *, cudaStream_t);
cudaError_t launch_reduce_partials(const double *partial, int k, int nchunk, double *out, cudaStream_t s,
                                   HostValue *pub, int32_t seq, double *root_a, double *root_b) {
    reduce_partials_kernel<<<k, 256, 0, s>>>(partial, nchunk, out, pub, seq, root_a, root_b);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_multi_axpy(T *w, const T *V, size_t ld, int k, const double *coef, double sign, size_t n,
                              cudaStream_t s) {
    multi_axpy_kernel_go<T>(blocks(n, 256), 256, 0, s, w, V, ld, k, coef, sign, n);
    return cudaGetLastError();
}
cudaError_t launch_scale_round(const double *w, const double *hnext, double *v64, float *v32, size_t n,
                               cudaStream_t s) {
    scale_round_kernel<<<blocks(n, 256), 256, 0, s>>>(w, hnext, v64, v32, n);
    return cudaGetLastError();
}
cudaError_t launch_widen(const float *a, double *b, size_t n, cudaStream_t s) {
    widen_kernel<<<blocks(n, 256), 256, 0, s>>>(a, b, n);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_scale_copy(const T *w, T *v, const double *denom, size_t n, cudaStream_t s) {
    scale_copy_kernel_go<T>(blocks(n, 256), 256, 0, s, w, v, denom, n);
    return cudaGetLastError();
}
cudaError_t launch_hessenberg_solve(const double *Hm, int ldh, const double *sv, int k, double *y, cudaStream_t s) {
    hessenberg_solve_kernel_go(1, 128, 0, s, Hm, ldh, sv, k, y);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_fill(T *x, T v, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    fill_kernel_go<T>(blocks(n, 256), 256, 0, s, x, v, n);
    return cudaGetLastError();
}
cudaError_t launch_d2f_norm(const double *x, float *y, float *z, const double *scale, size_t n, double *partial,
                            int nchunk, unsigned int *counter, double *out, double *root_a, double *root_b,
                            cudaStream_t s) {
    d2f_norm_kernel_go(unsigned(nchunk), 256, 0, s, x, y, z, scale, n, partial, counter, out, root_a, root_b);
    return cudaGetLastError();
}
cudaError_t launch_d2f_scaled(const double *x, float *y, const double *scale, size_t n, cudaStream_t s) {
    d2f_scaled_kernel_go(blocks(n, 256), 256, 0, s, x, y, scale, n);
    return cudaGetLastError();
}


template <typename T>
cudaError_t launch_gs_step(const T *V, size_t ld, int j, T *w, double *partial, unsigned int *counter, int nblk,
                           double *h1, double *h2, double *nrm2, double *Hm, int ldh, double *cs, double *sn,
                           double *sv, const double *bnorm, ReadBack *rb, ReadBack *host_rb, T *vnext, bool reorth, bool scale,
                           cudaStream_t s) {
    // h1 = V^T w comes with w from the operator kernel (apply_dots_kernel)
    const int k = j + 1;
    if (reorth) gs_update_dots_kernel<T><<<nblk, 256, 0, s>>>(V, ld, k, w, ld, h1, partial, counter, h2);
    gs_update_norm_givens_kernel_go<T>(nblk, 256, 0, s, V, ld, k, w, ld, h1, reorth ? h2 : nullptr, partial, counter,
                                                        nrm2, Hm, ldh, cs, sn, sv, j, bnorm, rb, host_rb);
    if (scale) {   // otherwise the next step's first smoothing sweep forms v_{j+1}
        const size_t n4 = ld / (16 / sizeof(T));
        gs_scale_kernel_go<T>(blocks(n4, 256), 256, 0, s, w, vnext, ld, rb);
    }
    return cudaGetLastError();
}
template cudaError_t launch_gs_step<float>(const float *, size_t, int, float *, double *, unsigned int *, int, double *,
                                           double *, double *, double *, int, double *, double *, double *,
                                           const double *, ReadBack *, ReadBack *, float *, bool, bool, cudaStream_t);
template cudaError_t launch_gs_step<double>(const double *, size_t, int, double *, double *, unsigned int *, int,
                                            double *, double *, double *, double *, int, double *, double *, double *,
                                            const double *, ReadBack *, ReadBack *, double *, bool, bool, cudaStream_t);

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
