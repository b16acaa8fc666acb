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

#include <cuda_bf16.h>
#include <type_traits>

namespace hdg {

// launch family of this file for pdl_launch (facet-row kernels)
constexpr unsigned kPdlFamily = 1;

namespace {

template <typename TO> __device__ __forceinline__ TO convert_to(double v);
template <> __device__ __forceinline__ double convert_to<double>(double v) { return v; }
template <> __device__ __forceinline__ float convert_to<float>(double v) { return float(v); }
template <> __device__ __forceinline__ __nv_bfloat16 convert_to<__nv_bfloat16>(double v) { return __double2bfloat16(v); }

// Operator values are packed in 16-byte groups: element j of facet e lives at
// group (j / G, e), lane j % G, with G = 16 / sizeof(storage); every thread
// issues one 16-byte load per group.  Storage FP64 (G = 2), FP32 (G = 4) or
// BF16 (G = 8, unpacked to FP32); arithmetic in the compute type T.
template <typename ST> struct Pack;
template <> struct Pack<double> {
    static constexpr int G = 2;
    using V = double2;
    __device__ static void unpack(const V &v, double (&o)[2]) { o[0] = v.x; o[1] = v.y; }
};
template <> struct Pack<float> {
    static constexpr int G = 4;
    using V = float4;
    __device__ static void unpack(const V &v, float (&o)[4]) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
};
template <> struct Pack<__nv_bfloat16> {
    static constexpr int G = 8;
    using V = uint4;
    __device__ static void unpack(const V &v, float (&o)[8]) {
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            o[2 * k] = __uint_as_float(w[k] << 16);
            o[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
        }
    }
};
template <typename ST> using unpacked_t = typename std::conditional<std::is_same<ST, double>::value, double, float>::type;

// gather the p+1 trace values of the facet and its four neighbours
template <int P, typename T>
__device__ __forceinline__ void gather_x(const int32_t *__restrict__ nbr, const T *__restrict__ x, int e, size_t NF,
                                         T (&xs)[5][P + 1]) {
    int src[5];
    src[0] = e;
#pragma unroll
    for (int b = 1; b < 5; ++b) src[b] = __ldg(nbr + size_t(b - 1) * NF + e);
#pragma unroll
    for (int b = 0; b < 5; ++b)
#pragma unroll
        for (int c = 0; c < P + 1; ++c) xs[b][c] = x[size_t(c) * NF + src[b]];
}

// y_r = sum_{b,c} S[(r*5+b)*PP+c] xs[b][c] with packed loads
template <int P, typename T, typename ST>
__device__ __forceinline__ void facet_rows_packed(const ST *__restrict__ Sval, int e, size_t NF,
                                                  const T (&xs)[5][P + 1], T (&y)[P + 1]) {
    constexpr int PP = P + 1, NS = 5 * PP * PP, G = Pack<ST>::G, NQ = (NS + G - 1) / G;
    using V = typename Pack<ST>::V;
    const V *Sp = reinterpret_cast<const V *>(Sval);
#pragma unroll
    for (int r = 0; r < PP; ++r) y[r] = T(0);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const V v = __ldg(Sp + size_t(q) * NF + e);
        unpacked_t<ST> o[G];
        Pack<ST>::unpack(v, o);
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int j = q * G + g;
            if (j < NS) {
                const int r = j / (5 * PP), rem = j % (5 * PP), b = rem / PP, c = rem % PP;
                y[r] = fma(T(o[g]), xs[b][c], y[r]);
            }
        }
    }
}

// out_r = sum_c Dinv[r*PP+c] v_c with packed loads
template <int P, typename T, typename DT>
__device__ __forceinline__ void block_solve_packed(const DT *__restrict__ Dinv, int e, size_t NF, const T (&v)[P + 1],
                                                   T (&out)[P + 1]) {
    constexpr int PP = P + 1, ND = PP * PP, G = Pack<DT>::G, NQ = (ND + G - 1) / G;
    using V = typename Pack<DT>::V;
    const V *Dp = reinterpret_cast<const V *>(Dinv);
#pragma unroll
    for (int r = 0; r < PP; ++r) out[r] = T(0);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const V w = __ldg(Dp + size_t(q) * NF + e);
        unpacked_t<DT> o[G];
        Pack<DT>::unpack(w, o);
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int j = q * G + g;
            if (j < ND) out[j / PP] = fma(T(o[g]), v[j % PP], out[j / PP]);
        }
    }
}

// FP32 facet-row kernels are bound by memory latency: cap registers so six
// 256-thread blocks fit per SM (one wave over the facets of large meshes);
// FP64 ones are bound by the FP64 pipe and keep their registers.
template <typename T> struct MinBlocks { static constexpr int value = sizeof(T) == 4 ? 6 : 1; };
// the operator kernel with the Gram-Schmidt dots: as above for FP32 (one wave),
// four blocks per SM for FP64
template <typename T> struct DotsMinBlocks { static constexpr int value = sizeof(T) == 4 ? 6 : 4; };

template <int P, typename T, typename ST>
__global__ void __launch_bounds__(256, MinBlocks<T>::value) apply_kernel(int NF, const ST *__restrict__ Sval, const int32_t *__restrict__ nbr,
                                                    const T *__restrict__ x, T *__restrict__ y) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NF) return;
    T xs[5][P + 1], v[P + 1];
    gather_x<P, T>(nbr, x, e, NF, xs);
    facet_rows_packed<P, T, ST>(Sval, e, NF, xs, v);
#pragma unroll
    for (int r = 0; r <= P; ++r) y[size_t(r) * NF + e] = v[r];
}

// y = S x (as apply_kernel) and h = V^T y over the first k basis vectors (the
// first Gram-Schmidt pass of an Arnoldi step): each block sums its facets'
// rows, four vectors at a time, into per-block partials; the last block to
// finish adds the partials in block order (deterministic) into h.
template <int P, typename T, typename ST>
__device__ __forceinline__ void apply_dots_kernel_impl(int bid_, int nb_, int NF, const ST *__restrict__ Sval,
                                                       const int32_t *__restrict__ nbr, const T *__restrict__ x,
                                                       T *__restrict__ y, const T *__restrict__ V, size_t ld, int k,
                                                       double *__restrict__ partial,
                                                       unsigned int *__restrict__ counter, double *__restrict__ h) {
    using A = typename std::conditional<std::is_same<T, double>::value, double, float>::type;
    constexpr int PP = P + 1, G = 4;
    __shared__ A red[G][8];
    __shared__ bool last;
    const int e = bid_ * blockDim.x + threadIdx.x;
    const bool valid = e < NF;
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nwarp = blockDim.x / 32;
    T v[PP];
    if (valid) {
        T xs[5][PP];
        gather_x<P, T>(nbr, x, e, NF, xs);
        facet_rows_packed<P, T, ST>(Sval, e, NF, xs, v);
#pragma unroll
        for (int r = 0; r < PP; ++r) y[size_t(r) * NF + e] = v[r];
    } else {
#pragma unroll
        for (int r = 0; r < PP; ++r) v[r] = T(0);
    }
    for (int i0 = 0; i0 < k; i0 += G) {
        A acc[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            A a = A(0);
            if (valid && i0 + g < k) {
#pragma unroll
                for (int r = 0; r < PP; ++r) a = fma(A(V[size_t(i0 + g) * ld + size_t(r) * NF + e]), A(v[r]), a);
            }
            acc[g] = a;
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            A t = acc[g];
            for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
            if (lane == 0) red[g][warp] = t;
        }
        __syncthreads();
        if (threadIdx.x < G && i0 + int(threadIdx.x) < k) {
            A t = A(0);
            for (int q = 0; q < nwarp; ++q) t += red[threadIdx.x][q];
            partial[size_t(i0 + threadIdx.x) * nb_ + bid_] = double(t);
        }
        __syncthreads();
    }
    if (threadIdx.x < G) __threadfence();      // the writers' partials are visible before the count
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == nb_ - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    finish_partials(partial, int(nb_), k, h);
    if (threadIdx.x == 0) *counter = 0u;
}
template <int P, typename T, typename ST>
__global__ void __launch_bounds__(256, DotsMinBlocks<T>::value) apply_dots_kernel(int NF, const ST *__restrict__ Sval,
                                                            const int32_t *__restrict__ nbr, const T *__restrict__ x,
                                                            T *__restrict__ y, const T *__restrict__ V, size_t ld,
                                                            int k, double *__restrict__ partial,
                                                            unsigned int *__restrict__ counter,
                                                            double *__restrict__ h) {
    pdl_wait();
    apply_dots_kernel_impl<P, T, ST>(blockIdx.x, gridDim.x, NF, Sval, nbr, x, y, V, ld, k, partial, counter, h);
}
template <int P, typename T, typename ST>
struct apply_dots_kernel_args {
    int nb_;
    int NF;
    const ST *Sval;
    const int32_t *nbr;
    const T *x;
    T *y;
    const T *V;
    size_t ld;
    int k;
    double *partial;
    unsigned int *counter;
    double *h;
};
template <int P, typename T, typename ST>
__global__ void __launch_bounds__(256, DotsMinBlocks<T>::value) apply_dots_kernel_multi(const __grid_constant__ MultiP<apply_dots_kernel_args<P, T, ST>> M) {
    pdl_wait();
    int b_;
    const apply_dots_kernel_args<P, T, ST> &q_ = M.a[merge_find(M.start, M.n, b_)];
    apply_dots_kernel_impl<P, T, ST>(b_, q_.nb_, q_.NF, q_.Sval, q_.nbr, q_.x, q_.y, q_.V, q_.ld, q_.k, q_.partial,
        q_.counter, q_.h);
}
template <int P, typename T, typename ST>
void apply_dots_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, int NF, const ST *Sval,
                          const int32_t *nbr, const T *x, T *y, const T *V, size_t ld, int k, double *partial,
                          unsigned int *counter, double *h) {
    if (Recorder *r_ = batch_recorder()) {
        apply_dots_kernel_args<P, T, ST> q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.NF = NF;
        q_.Sval = Sval;
        q_.nbr = nbr;
        q_.x = x;
        q_.y = y;
        q_.V = V;
        q_.ld = ld;
        q_.k = k;
        q_.partial = partial;
        q_.counter = counter;
        q_.h = h;
        batch_record(r_, reinterpret_cast<const void *>(&apply_dots_kernel_multi<P, T, ST>), q_, grid_, block_, smem_, kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &apply_dots_kernel<P, T, ST>, grid_, block_, smem_, s_, NF, Sval, nbr, x, y, V, ld, k, partial, counter, h);
}


template <int P, typename T, typename ST>
__device__ __forceinline__ void residual_kernel_impl(int bid_, int nb_, int NF, const ST *__restrict__ Sval,
                                                     const int32_t *__restrict__ nbr, const T *__restrict__ b,
                                                     const T *__restrict__ x, T *__restrict__ res) {
    const int e = bid_ * blockDim.x + threadIdx.x;
    if (e >= NF) return;
    T xs[5][P + 1], v[P + 1];
    gather_x<P, T>(nbr, x, e, NF, xs);
    facet_rows_packed<P, T, ST>(Sval, e, NF, xs, v);
#pragma unroll
    for (int r = 0; r <= P; ++r) res[size_t(r) * NF + e] = b[size_t(r) * NF + e] - v[r];
}
template <int P, typename T, typename ST>
__global__ void __launch_bounds__(256, MinBlocks<T>::value) residual_kernel(int NF, const ST *__restrict__ Sval,
                                                                            const int32_t *__restrict__ nbr,
                                                                            const T *__restrict__ b,
                                                                            const T *__restrict__ x,
                                                                            T *__restrict__ res) {
    pdl_wait();
    residual_kernel_impl<P, T, ST>(blockIdx.x, gridDim.x, NF, Sval, nbr, b, x, res);
}
template <int P, typename T, typename ST>
struct residual_kernel_args {
    int nb_;
    int NF;
    const ST *Sval;
    const int32_t *nbr;
    const T *b;
    const T *x;
    T *res;
};
template <int P, typename T, typename ST>
__global__ void __launch_bounds__(256, MinBlocks<T>::value) residual_kernel_multi(const __grid_constant__ MultiP<residual_kernel_args<P, T, ST>> M) {
    pdl_wait();
    int b_;
    const residual_kernel_args<P, T, ST> &q_ = M.a[merge_find(M.start, M.n, b_)];
    residual_kernel_impl<P, T, ST>(b_, q_.nb_, q_.NF, q_.Sval, q_.nbr, q_.b, q_.x, q_.res);
}
template <int P, typename T, typename ST>
void residual_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, int NF, const ST *Sval,
                        const int32_t *nbr, const T *b, const T *x, T *res) {
    if (Recorder *r_ = batch_recorder()) {
        residual_kernel_args<P, T, ST> q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.NF = NF;
        q_.Sval = Sval;
        q_.nbr = nbr;
        q_.b = b;
        q_.x = x;
        q_.res = res;
        batch_record(r_, reinterpret_cast<const void *>(&residual_kernel_multi<P, T, ST>), q_, grid_, block_, smem_, kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &residual_kernel<P, T, ST>, grid_, block_, smem_, s_, NF, Sval, nbr, b, x, res);
}


// One sweep x_out = x + omega D_e^-1 (b - S x)_e; with CHEB, a step of the
// Chebyshev iteration x_out = x + omega D_e^-1 (b - S x)_e + beta (x - x_prev)
// (x_prev null: the previous iterate is zero).  x_out may alias x_prev: each
// thread reads x_prev only at its own facet before writing it.
template <int P, typename T, typename ST, bool CHEB = false>
__device__ __forceinline__ void smooth_kernel_impl(int bid_, int nb_, int NF, const ST *__restrict__ Sval,
                                                   const T *__restrict__ Dinv, const int32_t *__restrict__ nbr,
                                                   const T *__restrict__ b, const T *__restrict__ x, T *xout, T omega,
                                                   T beta, const T *xprev) {
    constexpr int PP = P + 1;
    const int e = bid_ * blockDim.x + threadIdx.x;
    if (e >= NF) return;
    T xs[5][PP], v[PP], d[PP];
    gather_x<P, T>(nbr, x, e, NF, xs);
    facet_rows_packed<P, T, ST>(Sval, e, NF, xs, v);
#pragma unroll
    for (int r = 0; r < PP; ++r) v[r] = b[size_t(r) * NF + e] - v[r];
    block_solve_packed<P, T, T>(Dinv, e, NF, v, d);
    if constexpr (CHEB) {
#pragma unroll
        for (int r = 0; r < PP; ++r) {
            const T xp = xprev ? xprev[size_t(r) * NF + e] : T(0);
            xout[size_t(r) * NF + e] = fma(beta, xs[0][r] - xp, fma(omega, d[r], xs[0][r]));
        }
    } else {
#pragma unroll
        for (int r = 0; r < PP; ++r) xout[size_t(r) * NF + e] = fma(omega, d[r], xs[0][r]);
    }
}
template <int P, typename T, typename ST, bool CHEB = false>
__global__ void __launch_bounds__(256, MinBlocks<T>::value) smooth_kernel(int NF, const ST *__restrict__ Sval,
                                                                          const T *__restrict__ Dinv,
                                                                          const int32_t *__restrict__ nbr,
                                                                          const T *__restrict__ b,
                                                                          const T *__restrict__ x, T *xout, T omega,
                                                                          T beta, const T *xprev) {
    pdl_wait();
    smooth_kernel_impl<P, T, ST, CHEB>(blockIdx.x, gridDim.x, NF, Sval, Dinv, nbr, b, x, xout, omega, beta, xprev);
}
template <int P, typename T, typename ST, bool CHEB = false>
struct smooth_kernel_args {
    int nb_;
    int NF;
    const ST *Sval;
    const T *Dinv;
    const int32_t *nbr;
    const T *b;
    const T *x;
    T *xout;
    T omega;
    T beta;
    const T *xprev;
};
template <int P, typename T, typename ST, bool CHEB = false>
__global__ void __launch_bounds__(256, MinBlocks<T>::value) smooth_kernel_multi(const __grid_constant__ MultiP<smooth_kernel_args<P, T, ST, CHEB>> M) {
    pdl_wait();
    int b_;
    const smooth_kernel_args<P, T, ST, CHEB> &q_ = M.a[merge_find(M.start, M.n, b_)];
    smooth_kernel_impl<P, T, ST, CHEB>(b_, q_.nb_, q_.NF, q_.Sval, q_.Dinv, q_.nbr, q_.b, q_.x, q_.xout, q_.omega,
        q_.beta, q_.xprev);
}
template <int P, typename T, typename ST, bool CHEB = false>
void smooth_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, int NF, const ST *Sval,
                      const T *Dinv, const int32_t *nbr, const T *b, const T *x, T *xout, T omega, T beta,
                      const T *xprev) {
    if (Recorder *r_ = batch_recorder()) {
        smooth_kernel_args<P, T, ST, CHEB> q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.NF = NF;
        q_.Sval = Sval;
        q_.Dinv = Dinv;
        q_.nbr = nbr;
        q_.b = b;
        q_.x = x;
        q_.xout = xout;
        q_.omega = omega;
        q_.beta = beta;
        q_.xprev = xprev;
        batch_record(r_, reinterpret_cast<const void *>(&smooth_kernel_multi<P, T, ST, CHEB>), q_, grid_, block_, smem_, kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &smooth_kernel<P, T, ST, CHEB>, grid_, block_, smem_, s_, NF, Sval, Dinv, nbr, b, x, xout, omega, beta, xprev);
}


// First post-smoothing sweep with the coarse correction folded in:
// x' = x + pi e_c is formed on the fly for the five facets the rows touch,
// then x_out = x' + omega D_e^-1 (b - S x')_e.
// With X0, x' on the facet itself is also stored to x0out (the previous
// iterate of the Chebyshev step that follows).
template <int P, typename T, typename ST, bool X0 = false>
__device__ __forceinline__ void smooth_prolong_kernel_impl(int bid_, int nb_, int NF, const ST *__restrict__ Sval,
                                                           const T *__restrict__ Dinv,
                                                           const int32_t *__restrict__ nbr,
                                                           const int32_t *__restrict__ fverts,
                                                           const T *__restrict__ ec, const T *__restrict__ b,
                                                           const T *__restrict__ x, T *__restrict__ xout, T omega,
                                                           T *__restrict__ x0out) {
    constexpr int PP = P + 1;
    const int e = bid_ * blockDim.x + threadIdx.x;
    if (e >= NF) return;
    int src[5];
    src[0] = e;
#pragma unroll
    for (int bb = 1; bb < 5; ++bb) src[bb] = __ldg(nbr + size_t(bb - 1) * NF + e);
    T xs[5][PP], v[PP], d[PP];
#pragma unroll
    for (int bb = 0; bb < 5; ++bb) {
        const T lo = ec[__ldg(fverts + 2 * src[bb])], hi = ec[__ldg(fverts + 2 * src[bb] + 1)];
#pragma unroll
        for (int c = 0; c < PP; ++c) {
            const T t = T(c) / T(P);
            xs[bb][c] = x[size_t(c) * NF + src[bb]] + (T(1) - t) * lo + t * hi;
        }
    }
    facet_rows_packed<P, T, ST>(Sval, e, NF, xs, v);
#pragma unroll
    for (int r = 0; r < PP; ++r) v[r] = b[size_t(r) * NF + e] - v[r];
    block_solve_packed<P, T, T>(Dinv, e, NF, v, d);
#pragma unroll
    for (int r = 0; r < PP; ++r) xout[size_t(r) * NF + e] = fma(omega, d[r], xs[0][r]);
    if constexpr (X0) {
#pragma unroll
        for (int r = 0; r < PP; ++r) x0out[size_t(r) * NF + e] = xs[0][r];
    }
}
template <int P, typename T, typename ST, bool X0 = false>
__global__ void __launch_bounds__(256, MinBlocks<T>::value) smooth_prolong_kernel(int NF, const ST *__restrict__ Sval,
                                                                                  const T *__restrict__ Dinv,
                                                                                  const int32_t *__restrict__ nbr,
                                                                                  const int32_t *__restrict__ fverts,
                                                                                  const T *__restrict__ ec,
                                                                                  const T *__restrict__ b,
                                                                                  const T *__restrict__ x,
                                                                                  T *__restrict__ xout, T omega,
                                                                                  T *__restrict__ x0out) {
    pdl_wait();
    smooth_prolong_kernel_impl<P, T, ST, X0>(blockIdx.x, gridDim.x, NF, Sval, Dinv, nbr, fverts, ec, b, x, xout,
        omega, x0out);
}
template <int P, typename T, typename ST, bool X0 = false>
struct smooth_prolong_kernel_args {
    int nb_;
    int NF;
    const ST *Sval;
    const T *Dinv;
    const int32_t *nbr;
    const int32_t *fverts;
    const T *ec;
    const T *b;
    const T *x;
    T *xout;
    T omega;
    T *x0out;
};
template <int P, typename T, typename ST, bool X0 = false>
__global__ void __launch_bounds__(256, MinBlocks<T>::value) smooth_prolong_kernel_multi(const __grid_constant__ MultiP<smooth_prolong_kernel_args<P, T, ST, X0>> M) {
    pdl_wait();
    int b_;
    const smooth_prolong_kernel_args<P, T, ST, X0> &q_ = M.a[merge_find(M.start, M.n, b_)];
    smooth_prolong_kernel_impl<P, T, ST, X0>(b_, q_.nb_, q_.NF, q_.Sval, q_.Dinv, q_.nbr, q_.fverts, q_.ec, q_.b,
        q_.x, q_.xout, q_.omega, q_.x0out);
}
template <int P, typename T, typename ST, bool X0 = false>
void smooth_prolong_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, int NF, const ST *Sval,
                              const T *Dinv, const int32_t *nbr, const int32_t *fverts, const T *ec, const T *b,
                              const T *x, T *xout, T omega, T *x0out) {
    if (Recorder *r_ = batch_recorder()) {
        smooth_prolong_kernel_args<P, T, ST, X0> q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.NF = NF;
        q_.Sval = Sval;
        q_.Dinv = Dinv;
        q_.nbr = nbr;
        q_.fverts = fverts;
        q_.ec = ec;
        q_.b = b;
        q_.x = x;
        q_.xout = xout;
        q_.omega = omega;
        q_.x0out = x0out;
        batch_record(r_, reinterpret_cast<const void *>(&smooth_prolong_kernel_multi<P, T, ST, X0>), q_, grid_, block_, smem_, kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &smooth_prolong_kernel<P, T, ST, X0>, grid_, block_, smem_, s_, NF, Sval, Dinv, nbr, fverts, ec, b, x, xout,
        omega, x0out);
}


// first sweep from a zero initial guess: x = omega D^-1 b
template <int P, typename T>
__device__ __forceinline__ void smooth_first_kernel_impl(int bid_, int nb_, int NF, const T *__restrict__ Dinv,
                                                         const T *__restrict__ b, T *__restrict__ xout, T omega,
                                                         const T *__restrict__ w, const double *__restrict__ hnext,
                                                         T *__restrict__ bout) {
    // with w: the right-hand side is the next Arnoldi vector b = w / h_{j+1,j}
    // (the last Gram-Schmidt step of the previous iteration), also stored to
    // bout; the FP64 reciprocal is formed once per block
    __shared__ double inv_h;
    if (w != nullptr) {
        if (threadIdx.x == 0) inv_h = 1.0 / hnext[0];
        __syncthreads();
    }
    constexpr int PP = P + 1;
    const int e = bid_ * blockDim.x + threadIdx.x;
    if (e >= NF) return;
    T v[PP], d[PP];
    if (w != nullptr) {
        const T inv = T(inv_h);
#pragma unroll
        for (int c = 0; c < PP; ++c) {
            v[c] = w[size_t(c) * NF + e] * inv;
            bout[size_t(c) * NF + e] = v[c];
        }
    } else {
#pragma unroll
        for (int c = 0; c < PP; ++c) v[c] = b[size_t(c) * NF + e];
    }
    block_solve_packed<P, T, T>(Dinv, e, NF, v, d);
#pragma unroll
    for (int r = 0; r < PP; ++r) xout[size_t(r) * NF + e] = omega * d[r];
}
template <int P, typename T>
__global__ void smooth_first_kernel(int NF, const T *__restrict__ Dinv, const T *__restrict__ b, T *__restrict__ xout,
                                    T omega, const T *__restrict__ w, const double *__restrict__ hnext,
                                    T *__restrict__ bout) {
    pdl_wait();
    smooth_first_kernel_impl<P, T>(blockIdx.x, gridDim.x, NF, Dinv, b, xout, omega, w, hnext, bout);
}
template <int P, typename T>
struct smooth_first_kernel_args {
    int nb_;
    int NF;
    const T *Dinv;
    const T *b;
    T *xout;
    T omega;
    const T *w;
    const double *hnext;
    T *bout;
};
template <int P, typename T>
__global__ void smooth_first_kernel_multi(const __grid_constant__ MultiP<smooth_first_kernel_args<P, T>> M) {
    pdl_wait();
    int b_;
    const smooth_first_kernel_args<P, T> &q_ = M.a[merge_find(M.start, M.n, b_)];
    smooth_first_kernel_impl<P, T>(b_, q_.nb_, q_.NF, q_.Dinv, q_.b, q_.xout, q_.omega, q_.w, q_.hnext, q_.bout);
}
template <int P, typename T>
void smooth_first_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, int NF, const T *Dinv,
                            const T *b, T *xout, T omega, const T *w, const double *hnext, T *bout) {
    if (Recorder *r_ = batch_recorder()) {
        smooth_first_kernel_args<P, T> q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.NF = NF;
        q_.Dinv = Dinv;
        q_.b = b;
        q_.xout = xout;
        q_.omega = omega;
        q_.w = w;
        q_.hnext = hnext;
        q_.bout = bout;
        batch_record(r_, reinterpret_cast<const void *>(&smooth_first_kernel_multi<P, T>), q_, grid_, block_, smem_, kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &smooth_first_kernel<P, T>, grid_, block_, smem_, s_, NF, Dinv, b, xout, omega, w, hnext, bout);
}


// Repack the FP64 operator (groups of 2) into another storage precision
// (groups of 16 / sizeof(TO)); padding lanes are zero.
template <typename TO>
__global__ void repack_kernel(const double *__restrict__ src, int ns, size_t NF, TO *__restrict__ dst) {
    constexpr int G = 16 / int(sizeof(TO));
    const size_t tid = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const size_t nq = (size_t(ns) + G - 1) / G;
    if (tid >= nq * NF) return;
    const size_t q = tid / NF, e = tid % NF;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const size_t j = q * G + g;
        double v = 0.0;
        if (j < size_t(ns)) v = src[((j / 2) * NF + e) * 2 + (j % 2)];
        dst[(q * NF + e) * G + g] = convert_to<TO>(v);
    }
}

// lambda layout [NF][PP] <-> internal [PP][NF]
__global__ void to_internal_kernel(int NF, int PP, const double *ext, double *in) {
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= size_t(NF) * PP) return;
    const size_t e = i / PP, r = i % PP;
    in[r * NF + e] = ext[i];
}
__device__ __forceinline__ void to_external_kernel_impl(int bid_, int nb_, int NF, int PP, const double *in,
                                                        double *ext) {
    const size_t i = size_t(bid_) * blockDim.x + threadIdx.x;
    if (i >= size_t(NF) * PP) return;
    const size_t e = i / PP, r = i % PP;
    ext[i] = in[r * NF + e];
}
__global__ void to_external_kernel(int NF, int PP, const double *in, double *ext) {
    pdl_wait();
    to_external_kernel_impl(blockIdx.x, gridDim.x, NF, PP, in, ext);
}
struct to_external_kernel_args {
    int nb_;
    int NF;
    int PP;
    const double *in;
    double *ext;
};
__global__ void to_external_kernel_multi(const __grid_constant__ MultiP<to_external_kernel_args> M) {
    pdl_wait();
    int b_;
    const to_external_kernel_args &q_ = M.a[merge_find(M.start, M.n, b_)];
    to_external_kernel_impl(b_, q_.nb_, q_.NF, q_.PP, q_.in, q_.ext);
}
void to_external_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, int NF, int PP,
                           const double *in, double *ext) {
    if (Recorder *r_ = batch_recorder()) {
        to_external_kernel_args q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.NF = NF;
        q_.PP = PP;
        q_.in = in;
        q_.ext = ext;
        batch_record(r_, reinterpret_cast<const void *>(&to_external_kernel_multi), q_, grid_, block_, smem_, kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &to_external_kernel, grid_, block_, smem_, s_, NF, PP, in, ext);
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
// sum of a double over the block (fixed tree: warp shuffles, then warp 0 over
// the warp sums); thread 0 holds the block's sum
__device__ __forceinline__ double gather_block_sum(double v) {
    __shared__ double red[32];
    __syncthreads();
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

// g on facet e = the two cells' contributions (step 1 of Sec. 4.2); with
// partial non-null also ||g||^2 (block sums, the last block adding them in
// block order into out[0] and handing the value to the host through pub)
template <int P>
__device__ __forceinline__ void rhs_gather_kernel_impl(int bid_, int nb_, int N, int NF,
                                                       const double *__restrict__ ycell,
                                                       const int32_t *__restrict__ fcell,
                                                       const int32_t *__restrict__ fedge,
                                                       const int32_t *__restrict__ flip, double *__restrict__ g,
                                                       double *partial, unsigned int *counter, double *out,
                                                       HostValue *pub, int32_t seq, const F32Copy c32) {
    constexpr int PP = P + 1;
    const int e = bid_ * blockDim.x + threadIdx.x;
    double sq = 0.0;
    if (e < NF) {
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
        for (int r = 0; r < PP; ++r) {
            g[size_t(r) * NF + e] = v[r];
            sq = fma(v[r], v[r], sq);
        }
        if (c32.b32) {
#pragma unroll
            for (int r = 0; r < PP; ++r) {
                c32.b32[size_t(r) * NF + e] = float(v[r] * c32.scale);
                c32.z32[size_t(r) * NF + e] = 0.0f;
            }
        }
    }
    if (!partial) return;
    __shared__ bool last;
    const double tot = gather_block_sum(sq);
    if (threadIdx.x == 0) {
        partial[bid_] = tot;
        __threadfence();                       // the partial is visible before the count
        last = atomicAdd(counter, 1u) == unsigned(nb_) - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double a = 0.0;
    for (int i = threadIdx.x; i < nb_; i += blockDim.x) a += partial[i];
    a = gather_block_sum(a);
    if (threadIdx.x == 0) {
        *counter = 0u;
        out[0] = a;
        if (c32.root_a) *c32.root_a = sqrt(a) * c32.scale;
        if (c32.root_b) *c32.root_b = sqrt(a) * c32.scale;
        if (pub) {
            pub->v = a;
            __threadfence_system();
            *reinterpret_cast<volatile int32_t *>(&pub->seq) = seq;
        }
    }
}
template <int P>
__global__ void rhs_gather_kernel(int N, int NF, const double *__restrict__ ycell, const int32_t *__restrict__ fcell,
                                  const int32_t *__restrict__ fedge, const int32_t *__restrict__ flip,
                                  double *__restrict__ g, double *partial, unsigned int *counter, double *out,
                                  HostValue *pub, int32_t seq, const F32Copy c32) {
    pdl_wait();
    rhs_gather_kernel_impl<P>(blockIdx.x, gridDim.x, N, NF, ycell, fcell, fedge, flip, g, partial, counter, out, pub,
                              seq, c32);
}
template <int P>
struct rhs_gather_kernel_args {
    int nb_;
    int N;
    int NF;
    const double *ycell;
    const int32_t *fcell;
    const int32_t *fedge;
    const int32_t *flip;
    double *g;
    double *partial;
    unsigned int *counter;
    double *out;
    HostValue *pub;
    int32_t seq;
    F32Copy c32;
};
template <int P>
__global__ void rhs_gather_kernel_multi(const __grid_constant__ MultiP<rhs_gather_kernel_args<P>> M) {
    pdl_wait();
    int b_;
    const rhs_gather_kernel_args<P> &q_ = M.a[merge_find(M.start, M.n, b_)];
    rhs_gather_kernel_impl<P>(b_, q_.nb_, q_.N, q_.NF, q_.ycell, q_.fcell, q_.fedge, q_.flip, q_.g, q_.partial,
                              q_.counter, q_.out, q_.pub, q_.seq, q_.c32);
}
template <int P>
void rhs_gather_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, int N, int NF,
                          const double *ycell, const int32_t *fcell, const int32_t *fedge, const int32_t *flip,
                          double *g, double *partial, unsigned int *counter, double *out, HostValue *pub,
                          int32_t seq, const F32Copy &c32) {
    if (Recorder *r_ = batch_recorder()) {
        rhs_gather_kernel_args<P> q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.N = N;
        q_.NF = NF;
        q_.ycell = ycell;
        q_.fcell = fcell;
        q_.fedge = fedge;
        q_.flip = flip;
        q_.g = g;
        q_.partial = partial;
        q_.counter = counter;
        q_.out = out;
        q_.pub = pub;
        q_.seq = seq;
        q_.c32 = c32;
        batch_record(r_, reinterpret_cast<const void *>(&rhs_gather_kernel_multi<P>), q_, grid_, block_, smem_,
                     kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &rhs_gather_kernel<P>, grid_, block_, smem_, s_, N, NF, ycell, fcell, fedge, flip, g,
               partial, counter, out, pub, seq, c32);
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
__device__ __forceinline__ void restrict_kernel_impl(int bid_, int nb_, int nv, int NF,
                                                     const int32_t *__restrict__ v2f_ptr,
                                                     const int32_t *__restrict__ v2f, const T *__restrict__ r,
                                                     T *__restrict__ rc, const T *__restrict__ dinv0, T omega,
                                                     T *__restrict__ x0) {
    const int v = bid_ * blockDim.x + threadIdx.x;
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
    // first damped Jacobi sweep of the P1 level from zero, fused (x0 may be null)
    if (x0) x0[v] = omega * dinv0[v] * acc;
}
template <int P, typename T>
__global__ void restrict_kernel(int nv, int NF, const int32_t *__restrict__ v2f_ptr, const int32_t *__restrict__ v2f,
                                const T *__restrict__ r, T *__restrict__ rc, const T *__restrict__ dinv0, T omega,
                                T *__restrict__ x0) {
    pdl_wait();
    restrict_kernel_impl<P, T>(blockIdx.x, gridDim.x, nv, NF, v2f_ptr, v2f, r, rc, dinv0, omega, x0);
}
template <int P, typename T>
struct restrict_kernel_args {
    int nb_;
    int nv;
    int NF;
    const int32_t *v2f_ptr;
    const int32_t *v2f;
    const T *r;
    T *rc;
    const T *dinv0;
    T omega;
    T *x0;
};
template <int P, typename T>
__global__ void restrict_kernel_multi(const __grid_constant__ MultiP<restrict_kernel_args<P, T>> M) {
    pdl_wait();
    int b_;
    const restrict_kernel_args<P, T> &q_ = M.a[merge_find(M.start, M.n, b_)];
    restrict_kernel_impl<P, T>(b_, q_.nb_, q_.nv, q_.NF, q_.v2f_ptr, q_.v2f, q_.r, q_.rc, q_.dinv0, q_.omega, q_.x0);
}
template <int P, typename T>
void restrict_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, int nv, int NF,
                        const int32_t *v2f_ptr, const int32_t *v2f, const T *r, T *rc, const T *dinv0, T omega,
                        T *x0) {
    if (Recorder *r_ = batch_recorder()) {
        restrict_kernel_args<P, T> q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.nv = nv;
        q_.NF = NF;
        q_.v2f_ptr = v2f_ptr;
        q_.v2f = v2f;
        q_.r = r;
        q_.rc = rc;
        q_.dinv0 = dinv0;
        q_.omega = omega;
        q_.x0 = x0;
        batch_record(r_, reinterpret_cast<const void *>(&restrict_kernel_multi<P, T>), q_, grid_, block_, smem_, kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &restrict_kernel<P, T>, grid_, block_, smem_, s_, nv, NF, v2f_ptr, v2f, r, rc, dinv0, omega, x0);
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


}  // namespace

// operator storage per use: FP64 path, FP32 Krylov operator, and the
// preconditioner's copy (BF16 in HDG_MIXED_BF16, else the FP32 one)
template <typename T> struct Ops;
template <> struct Ops<double> {
    static const double *S(hdg_handle *h, bool) { return h->d_Sval; }
    static const double *D(hdg_handle *h) { return h->d_Dinv; }
};
template <> struct Ops<float> {
    static const float *S(hdg_handle *h, bool) { return h->d_Sval32; }
    static const float *D(hdg_handle *h) { return h->d_Dinv32; }
};
inline bool bf16_pre(hdg_handle *h) { return h->prm.precision == HDG_MIXED_BF16 && h->d_Sval16; }

template <typename T>
cudaError_t launch_apply_dots_t(hdg_handle *h, const T *x, T *y, const T *V, size_t ld, int k, double *partial,
                                unsigned int *counter, double *hdots) {
    HDG_DISPATCH_PF(h->pf, T, (apply_dots_kernel_go<P, T, T>(blocks(h->NF, 256), 256, 0, h->stream, 
                             h->NF, Ops<T>::S(h, false), h->d_nbr, x, y, V, ld, k, partial, counter, hdots)));
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_apply_t(hdg_handle *h, const T *x, T *y) {
    HDG_DISPATCH_PF(h->pf, T, (apply_kernel<P, T, T><<<blocks(h->NF, h->bs_facet), h->bs_facet, 0, h->stream>>>(h->NF, Ops<T>::S(h, false), h->d_nbr, x, y)));
    return cudaGetLastError();
}
// residual / smoothing kernels serve the preconditioner (pre = true) or the
// Krylov residual (pre = false)
template <typename T>
cudaError_t launch_residual_t(hdg_handle *h, const T *b, const T *x, T *r, bool pre) {
    if constexpr (std::is_same<T, float>::value) if (pre && bf16_pre(h)) {
        HDG_DISPATCH_PF(h->pf, T, (residual_kernel_go<P, T, __nv_bfloat16>(blocks(h->NF, h->bs_facet), h->bs_facet, 0, h->stream, h->NF, h->d_Sval16, h->d_nbr, b, x, r)));
        return cudaGetLastError();
    }
    {
        HDG_DISPATCH_PF(h->pf, T, (residual_kernel_go<P, T, T>(blocks(h->NF, h->bs_facet), h->bs_facet, 0, h->stream, h->NF, Ops<T>::S(h, pre), h->d_nbr, b, x, r)));
    }
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_smooth_t(hdg_handle *h, const T *b, const T *x, T *xout) {
    const T om = T(h->prm.omega);
    if constexpr (std::is_same<T, float>::value) if (bf16_pre(h)) {
        HDG_DISPATCH_PF(h->pf, T, (smooth_kernel_go<P, T, __nv_bfloat16>(blocks(h->NF, h->bs_facet), h->bs_facet, 0, h->stream, h->NF, h->d_Sval16, Ops<T>::D(h), h->d_nbr, b, x, xout, om, T(0), nullptr)));
        return cudaGetLastError();
    }
    {
        HDG_DISPATCH_PF(h->pf, T, (smooth_kernel_go<P, T, T>(blocks(h->NF, h->bs_facet), h->bs_facet, 0, h->stream, h->NF, Ops<T>::S(h, true), Ops<T>::D(h), h->d_nbr, b, x, xout, om, T(0), nullptr)));
    }
    return cudaGetLastError();
}
// a step of the Chebyshev iteration: xout = x + omega D^-1 (b - S x) + beta (x - xprev)
template <typename T>
cudaError_t launch_smooth_cheb_t(hdg_handle *h, const T *b, const T *x, T *xout, double omega, double beta,
                                 const T *xprev) {
    if constexpr (std::is_same<T, float>::value) if (bf16_pre(h)) {
        HDG_DISPATCH_PF(h->pf, T, (smooth_kernel_go<P, T, __nv_bfloat16, true>(blocks(h->NF, h->bs_facet), h->bs_facet, 0, h->stream, h->NF, h->d_Sval16, Ops<T>::D(h), h->d_nbr, b, x, xout, T(omega), T(beta), xprev)));
        return cudaGetLastError();
    }
    {
        HDG_DISPATCH_PF(h->pf, T, (smooth_kernel_go<P, T, T, true>(blocks(h->NF, h->bs_facet), h->bs_facet, 0, h->stream, h->NF, Ops<T>::S(h, true), Ops<T>::D(h), h->d_nbr, b, x, xout, T(omega), T(beta), xprev)));
    }
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_smooth_first_t(hdg_handle *h, const T *b, T *x, const T *w, const double *hnext, T *bout,
                                  double omega) {
    const T om = T(omega > 0 ? omega : h->prm.omega);
    HDG_DISPATCH_PF(h->pf, T, (smooth_first_kernel_go<P, T>(blocks(h->NF, h->bs_facet), h->bs_facet, 0, h->stream, h->NF, Ops<T>::D(h), b, x, om, w, hnext, bout)));
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_restrict_t(hdg_handle *h, const T *r, T *rc, const T *dinv0, T omega, T *x0) {
    HDG_DISPATCH_P(h->p, (restrict_kernel_go<P, T>(blocks(h->nv, 256), 256, 0, h->stream, h->nv, h->NF, h->d_v2f_ptr, h->d_v2f, r, rc, dinv0, omega, x0)));
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_smooth_prolong_t(hdg_handle *h, const T *ec, const T *b, const T *x, T *xout, double omega,
                                    T *x0out) {
    const T om = T(omega > 0 ? omega : h->prm.omega);
    if constexpr (std::is_same<T, float>::value) if (bf16_pre(h)) {
        if (x0out) {
            HDG_DISPATCH_P(h->p, (smooth_prolong_kernel_go<P, T, __nv_bfloat16, true>(blocks(h->NF, h->bs_facet), h->bs_facet, 0, h->stream, h->NF, h->d_Sval16, Ops<T>::D(h), h->d_nbr, h->d_facet_verts, ec, b, x, xout, om, x0out)));
        } else {
            HDG_DISPATCH_P(h->p, (smooth_prolong_kernel_go<P, T, __nv_bfloat16>(blocks(h->NF, h->bs_facet), h->bs_facet, 0, h->stream, h->NF, h->d_Sval16, Ops<T>::D(h), h->d_nbr, h->d_facet_verts, ec, b, x, xout, om, nullptr)));
        }
        return cudaGetLastError();
    }
    if (x0out) {
        HDG_DISPATCH_P(h->p, (smooth_prolong_kernel_go<P, T, T, true>(blocks(h->NF, h->bs_facet), h->bs_facet, 0, h->stream, h->NF, Ops<T>::S(h, true), Ops<T>::D(h), h->d_nbr, h->d_facet_verts, ec, b, x, xout, om, x0out)));
    } else {
        HDG_DISPATCH_P(h->p, (smooth_prolong_kernel_go<P, T, T>(blocks(h->NF, h->bs_facet), h->bs_facet, 0, h->stream, h->NF, Ops<T>::S(h, true), Ops<T>::D(h), h->d_nbr, h->d_facet_verts, ec, b, x, xout, om, nullptr)));
    }
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_prolong_add_t(hdg_handle *h, const T *ec, T *x) {
    HDG_DISPATCH_P(h->p, (prolong_add_kernel<P, T><<<blocks(h->NF, h->bs_facet), h->bs_facet, 0, h->stream>>>(h->NF, h->d_facet_verts, ec, x)));
    return cudaGetLastError();
}

// FP32 / BF16 copies of the packed FP64 operator and the FP32 inverse blocks
cudaError_t launch_repack(hdg_handle *h) {
    const int pp = h->pp, ns = 5 * pp * pp, nd = pp * pp;
    const size_t NF = h->NF;
    auto nq = [&](int n, int G) { return (size_t(n) + G - 1) / G * NF; };
    if (h->d_Sval32) {
        repack_kernel<float><<<blocks(nq(ns, 4), 256), 256, 0, h->stream>>>(h->d_Sval, ns, NF, h->d_Sval32);
        repack_kernel<float><<<blocks(nq(nd, 4), 256), 256, 0, h->stream>>>(h->d_Dinv, nd, NF, h->d_Dinv32);
    }
    if (h->d_Sval16)
        repack_kernel<__nv_bfloat16><<<blocks(nq(ns, 8), 256), 256, 0, h->stream>>>(h->d_Sval, ns, NF, h->d_Sval16);
    return cudaGetLastError();
}

template cudaError_t launch_apply_t<double>(hdg_handle *, const double *, double *);
template cudaError_t launch_apply_dots_t<double>(hdg_handle *, const double *, double *, const double *, size_t, int,
                                                 double *, unsigned int *, double *);
template cudaError_t launch_apply_dots_t<float>(hdg_handle *, const float *, float *, const float *, size_t, int,
                                                double *, unsigned int *, double *);
template cudaError_t launch_apply_t<float>(hdg_handle *, const float *, float *);
template cudaError_t launch_residual_t<double>(hdg_handle *, const double *, const double *, double *, bool);
template cudaError_t launch_residual_t<float>(hdg_handle *, const float *, const float *, float *, bool);
template cudaError_t launch_smooth_t<double>(hdg_handle *, const double *, const double *, double *);
template cudaError_t launch_smooth_t<float>(hdg_handle *, const float *, const float *, float *);
template cudaError_t launch_smooth_cheb_t<double>(hdg_handle *, const double *, const double *, double *, double,
                                                  double, const double *);
template cudaError_t launch_smooth_cheb_t<float>(hdg_handle *, const float *, const float *, float *, double, double,
                                                 const float *);
template cudaError_t launch_smooth_first_t<double>(hdg_handle *, const double *, double *, const double *,
                                                   const double *, double *, double);
template cudaError_t launch_smooth_first_t<float>(hdg_handle *, const float *, float *, const float *, const double *,
                                                  float *, double);
template cudaError_t launch_restrict_t<double>(hdg_handle *, const double *, double *, const double *, double, double *);
template cudaError_t launch_restrict_t<float>(hdg_handle *, const float *, float *, const float *, float, float *);
template cudaError_t launch_smooth_prolong_t<double>(hdg_handle *, const double *, const double *, const double *, double *,
                                                     double, double *);
template cudaError_t launch_smooth_prolong_t<float>(hdg_handle *, const float *, const float *, const float *, float *,
                                                    double, float *);
template cudaError_t launch_prolong_add_t<double>(hdg_handle *, const double *, double *);
template cudaError_t launch_prolong_add_t<float>(hdg_handle *, const float *, float *);

cudaError_t launch_to_internal(hdg_handle *h, const double *ext, double *in) {
    size_t n = size_t(h->NF) * h->pp;
    to_internal_kernel<<<blocks(n, 256), 256, 0, h->stream>>>(h->NF, h->pp, ext, in);
    return cudaGetLastError();
}
cudaError_t launch_to_external(hdg_handle *h, const double *in, double *ext) {
    size_t n = size_t(h->NF) * h->pp;
    to_external_kernel_go(blocks(n, 256), 256, 0, h->stream, h->NF, h->pp, in, ext);
    return cudaGetLastError();
}

cudaError_t launch_rhs_gather(hdg_handle *h, const double *ycell, double *g, const NormOut &nrm) {
    HDG_DISPATCH_P(h->p, (rhs_gather_kernel_go<P>(blocks(h->NF, h->bs_facet), h->bs_facet, 0, h->stream, h->N, h->NF,
                                                  ycell, h->d_facet_cell, h->d_facet_edge, h->d_flip, g, nrm.partial,
                                                  nrm.counter, nrm.out, nrm.pub, nrm.seq, nrm.f32)));
    return cudaGetLastError();
}

cudaError_t launch_rhs(hdg_handle *h, const double *r_u, const double *r_h, double *g, double *ycell,
                       const NormOut &nrm) {
    if (h->prm.flux == 1) return nrm.partial ? cudaErrorInvalidValue : launch_rhs_lf(h, r_u, r_h, g, ycell);
    size_t n = size_t(h->N) * h->m;
    HDG_DISPATCH_P(h->p, (rhs_cell_kernel<P><<<blocks(n, 256), 256, 0, h->stream>>>(h->N, h->d_W, r_u, r_h, ycell)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_rhs_gather(h, ycell, g, nrm);
}

cudaError_t launch_recover(hdg_handle *h, const double *r_u, const double *r_h, const double *lam, double *u,
                           double *hout) {
    if (h->prm.flux == 1) return launch_recover_lf(h, r_u, r_h, lam, u, hout);
    size_t n = size_t(h->N) * h->nK;
    HDG_DISPATCH_P(h->p, (recover_kernel<P><<<blocks(n, 256), 256, 0, h->stream>>>(h->N, h->NF, h->d_Rm, h->d_Xb, r_u, r_h, lam, h->d_facet_of, h->d_flip, u, hout)));
    return cudaGetLastError();
}

}  // namespace hdg
