// Geometric V-cycle on the nested P1 levels for the coarse problem of the
// two-level method (Eq. coarse_problem_upwind): damped Jacobi smoothing with
// the level operators in padded row-major ELL form (width W a multiple of 4,
// slot q of row i at i * W + q), restriction by the transpose of the midpoint
// prolongation, and a dense inverse on the coarsest level.  A row's columns
// and values load as 16-byte vectors; its W products are summed in slot order.
// Three launch structures, all with that arithmetic: one kernel per step
// (large levels), patch kernels that recompute a one-ring halo so that a
// sweep and the step consuming it share a launch (mid-size levels), and one
// CTA for the small levels, staged from a pre-packed shared-memory image.
#include "common.h"

namespace hdg {

// launch family of this file for pdl_launch (P1 kernels)
constexpr unsigned kPdlFamily = 2;

namespace {

inline unsigned blocks(size_t n, int bs) { return unsigned((n + bs - 1) / bs); }

// x_out = x + omega D^-1 (b - A x); first sweep (x = 0): x_out = omega D^-1 b
// four consecutive values of a row as one 16-byte load (two for FP64)
__device__ __forceinline__ void load4(const float *p, float v[4]) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void load4(const double *p, double v[4]) {
    const double2 t0 = reinterpret_cast<const double2 *>(p)[0], t1 = reinterpret_cast<const double2 *>(p)[1];
    v[0] = t0.x; v[1] = t0.y; v[2] = t1.x; v[3] = t1.y;
}

// (A x)_i for a padded row-major ELL operator of width W (a multiple of 4)
template <typename T>
__device__ __forceinline__ T ell_row(int i, int W, const int32_t *__restrict__ col, const T *__restrict__ A,
                                     const T *__restrict__ x) {
    const int32_t *c = col + size_t(i) * W;
    const T *a = A + size_t(i) * W;
    T ax = T(0);
#pragma unroll 2
    for (int q = 0; q < W; q += 4) {
        const int4 cc = *reinterpret_cast<const int4 *>(c + q);
        T av[4];
        load4(a + q, av);
        ax = fma(av[0], x[cc.x], ax);
        ax = fma(av[1], x[cc.y], ax);
        ax = fma(av[2], x[cc.z], ax);
        ax = fma(av[3], x[cc.w], ax);
    }
    return ax;
}

template <typename T>
__device__ __forceinline__ void jacobi_kernel_impl(int bid_, int nb_, int n, int W, const int32_t *__restrict__ col,
                                                   const T *__restrict__ A, const T *__restrict__ dinv,
                                                   const T *__restrict__ b, const T *__restrict__ x,
                                                   T *__restrict__ xout, T omega, int first) {
    // the static row (operator values, columns, inverse diagonal) before the
    // wait for the previous kernel, the vectors after it
    const int i = bid_ * blockDim.x + threadIdx.x;
    const bool ok = i < n;
    T di = T(0), av[8];
    int cs[8];
    const bool pre = ok && !first && W == 8;
    if (ok) di = dinv[i];
    if (pre) {
        const int4 c0 = *reinterpret_cast<const int4 *>(col + size_t(i) * 8);
        const int4 c1 = *reinterpret_cast<const int4 *>(col + size_t(i) * 8 + 4);
        cs[0] = c0.x; cs[1] = c0.y; cs[2] = c0.z; cs[3] = c0.w;
        cs[4] = c1.x; cs[5] = c1.y; cs[6] = c1.z; cs[7] = c1.w;
        load4(A + size_t(i) * 8, av);
        load4(A + size_t(i) * 8 + 4, av + 4);
    }
    pdl_wait();
    if (!ok) return;
    if (first) {
        xout[i] = omega * di * b[i];
        return;
    }
    T ax = T(0);
    if (pre) {
#pragma unroll
        for (int q = 0; q < 8; ++q) ax = fma(av[q], x[cs[q]], ax);
    } else {
        ax = ell_row(i, W, col, A, x);
    }
    xout[i] = fma(omega * di, b[i] - ax, x[i]);
}
template <typename T>
__global__ void jacobi_kernel(int n, int W, const int32_t *__restrict__ col, const T *__restrict__ A,
                              const T *__restrict__ dinv, const T *__restrict__ b, const T *__restrict__ x,
                              T *__restrict__ xout, T omega, int first) {
    jacobi_kernel_impl<T>(blockIdx.x, gridDim.x, n, W, col, A, dinv, b, x, xout, omega, first);
}
template <typename T>
struct jacobi_kernel_args {
    int nb_;
    int n;
    int W;
    const int32_t *col;
    const T *A;
    const T *dinv;
    const T *b;
    const T *x;
    T *xout;
    T omega;
    int first;
};
template <typename T>
__global__ void jacobi_kernel_multi(const __grid_constant__ MultiP<jacobi_kernel_args<T>> M) {
    int b_;
    const jacobi_kernel_args<T> &q_ = M.a[merge_find(M.start, M.n, b_)];
    jacobi_kernel_impl<T>(b_, q_.nb_, q_.n, q_.W, q_.col, q_.A, q_.dinv, q_.b, q_.x, q_.xout, q_.omega, q_.first);
}
template <typename T>
void jacobi_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, int n, int W,
                      const int32_t *col, const T *A, const T *dinv, const T *b, const T *x, T *xout, T omega,
                      int first) {
    if (Recorder *r_ = batch_recorder()) {
        jacobi_kernel_args<T> q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.n = n;
        q_.W = W;
        q_.col = col;
        q_.A = A;
        q_.dinv = dinv;
        q_.b = b;
        q_.x = x;
        q_.xout = xout;
        q_.omega = omega;
        q_.first = first;
        batch_record(r_, reinterpret_cast<const void *>(&jacobi_kernel_multi<T>), q_, grid_, block_, smem_, kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &jacobi_kernel<T>, grid_, block_, smem_, s_, n, W, col, A, dinv, b, x, xout, omega, first);
}


template <typename T>
__device__ __forceinline__ void prolong_add_kernel_impl(int bid_, int nb_, int nf, const int32_t *__restrict__ parent,
                                                        const T *__restrict__ ec, T *__restrict__ xf) {
    const int i = bid_ * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    const int a = parent[2 * i], b = parent[2 * i + 1];
    xf[i] += (a == b) ? ec[a] : T(0.5) * (ec[a] + ec[b]);
}
template <typename T>
__global__ void prolong_add_kernel(int nf, const int32_t *__restrict__ parent, const T *__restrict__ ec,
                                   T *__restrict__ xf) {
    pdl_wait();
    prolong_add_kernel_impl<T>(blockIdx.x, gridDim.x, nf, parent, ec, xf);
}
template <typename T>
struct prolong_add_kernel_args {
    int nb_;
    int nf;
    const int32_t *parent;
    const T *ec;
    T *xf;
};
template <typename T>
__global__ void prolong_add_kernel_multi(const __grid_constant__ MultiP<prolong_add_kernel_args<T>> M) {
    pdl_wait();
    int b_;
    const prolong_add_kernel_args<T> &q_ = M.a[merge_find(M.start, M.n, b_)];
    prolong_add_kernel_impl<T>(b_, q_.nb_, q_.nf, q_.parent, q_.ec, q_.xf);
}
template <typename T>
void prolong_add_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, int nf,
                           const int32_t *parent, const T *ec, T *xf) {
    if (Recorder *r_ = batch_recorder()) {
        prolong_add_kernel_args<T> q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.nf = nf;
        q_.parent = parent;
        q_.ec = ec;
        q_.xf = xf;
        batch_record(r_, reinterpret_cast<const void *>(&prolong_add_kernel_multi<T>), q_, grid_, block_, smem_, kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &prolong_add_kernel<T>, grid_, block_, smem_, s_, nf, parent, ec, xf);
}




// Going down one level, fused: b_c = R (b_f - A_f x_f) with the fine residual
// formed on the fly for each child, and the first pre-smoothing sweep of the
// coarse level from zero, x_c = omega D_c^-1 b_c (skipped when xc is null).
// Eight lanes per coarse vertex share its children; their partial sums are
// combined by a fixed shuffle tree (deterministic).
template <typename T>
__device__ __forceinline__ void down_kernel_impl(int bid_, int nb_, int nc, const int32_t *__restrict__ cp,
                                                 const int32_t *__restrict__ ci, const T *__restrict__ cw, int nf,
                                                 int W, const int32_t *__restrict__ col, const T *__restrict__ A,
                                                 const T *__restrict__ bf, const T *__restrict__ xf,
                                                 const T *__restrict__ dinv_c, T omega, T *__restrict__ bc,
                                                 T *__restrict__ xc) {
    const int gid = (bid_ * blockDim.x + threadIdx.x) >> 3, lane = threadIdx.x & 7;
    const bool valid = gid < nc;
    // the lane's first child row (static: index, weight, columns, values)
    // before the wait for the previous kernel, the vectors after it
    int k0 = 0, k1 = 0, f0 = 0, cs[8];
    T w0 = T(0), av[8];
    bool pre = false;
    if (valid) {
        k0 = cp[gid] + lane;
        k1 = cp[gid + 1];
        if (k0 < k1 && W == 8) {
            pre = true;
            f0 = ci[k0];
            w0 = cw[k0];
            const int4 c0 = *reinterpret_cast<const int4 *>(col + size_t(f0) * 8);
            const int4 c1 = *reinterpret_cast<const int4 *>(col + size_t(f0) * 8 + 4);
            cs[0] = c0.x; cs[1] = c0.y; cs[2] = c0.z; cs[3] = c0.w;
            cs[4] = c1.x; cs[5] = c1.y; cs[6] = c1.z; cs[7] = c1.w;
            load4(A + size_t(f0) * 8, av);
            load4(A + size_t(f0) * 8 + 4, av + 4);
        }
    }
    pdl_wait();
    T acc = T(0);
    if (valid) {
        int k = k0;
        if (pre) {
            T ax = T(0);
#pragma unroll
            for (int q = 0; q < 8; ++q) ax = fma(av[q], xf[cs[q]], ax);
            acc = fma(w0, bf[f0] - ax, acc);
            k += 8;
        }
        for (; k < k1; k += 8) {
            const int f = ci[k];
            acc = fma(cw[k], bf[f] - ell_row(f, W, col, A, xf), acc);
        }
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 4);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    if (valid && lane == 0) {
        bc[gid] = acc;
        if (xc) xc[gid] = omega * dinv_c[gid] * acc;
    }
}
template <typename T>
__global__ void __launch_bounds__(256) down_kernel(int nc, const int32_t *__restrict__ cp,
                                                   const int32_t *__restrict__ ci, const T *__restrict__ cw, int nf,
                                                   int W, const int32_t *__restrict__ col, const T *__restrict__ A,
                                                   const T *__restrict__ bf, const T *__restrict__ xf,
                                                   const T *__restrict__ dinv_c, T omega, T *__restrict__ bc,
                                                   T *__restrict__ xc) {
    down_kernel_impl<T>(blockIdx.x, gridDim.x, nc, cp, ci, cw, nf, W, col, A, bf, xf, dinv_c, omega, bc, xc);
}
template <typename T>
struct down_kernel_args {
    int nb_;
    int nc;
    const int32_t *cp;
    const int32_t *ci;
    const T *cw;
    int nf;
    int W;
    const int32_t *col;
    const T *A;
    const T *bf;
    const T *xf;
    const T *dinv_c;
    T omega;
    T *bc;
    T *xc;
};
template <typename T>
__global__ void __launch_bounds__(256) down_kernel_multi(const __grid_constant__ MultiP<down_kernel_args<T>> M) {
    int b_;
    const down_kernel_args<T> &q_ = M.a[merge_find(M.start, M.n, b_)];
    down_kernel_impl<T>(b_, q_.nb_, q_.nc, q_.cp, q_.ci, q_.cw, q_.nf, q_.W, q_.col, q_.A, q_.bf, q_.xf, q_.dinv_c,
        q_.omega, q_.bc, q_.xc);
}
template <typename T>
void down_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, int nc, const int32_t *cp,
                    const int32_t *ci, const T *cw, int nf, int W, const int32_t *col, const T *A, const T *bf,
                    const T *xf, const T *dinv_c, T omega, T *bc, T *xc) {
    if (Recorder *r_ = batch_recorder()) {
        down_kernel_args<T> q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.nc = nc;
        q_.cp = cp;
        q_.ci = ci;
        q_.cw = cw;
        q_.nf = nf;
        q_.W = W;
        q_.col = col;
        q_.A = A;
        q_.bf = bf;
        q_.xf = xf;
        q_.dinv_c = dinv_c;
        q_.omega = omega;
        q_.bc = bc;
        q_.xc = xc;
        batch_record(r_, reinterpret_cast<const void *>(&down_kernel_multi<T>), q_, grid_, block_, smem_, kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &down_kernel<T>, grid_, block_, smem_, s_, nc, cp, ci, cw, nf, W, col, A, bf, xf, dinv_c, omega, bc, xc);
}


// Going up one level, fused: x' = x + P e_c (midpoint prolongation, formed on
// the fly for every column) followed by one damped Jacobi sweep on x'.
template <typename T>
__device__ __forceinline__ void up_kernel_impl(int bid_, int nb_, int nf, int W, const int32_t *__restrict__ col,
                                               const T *__restrict__ A, const T *__restrict__ dinv,
                                               const T *__restrict__ b, const T *__restrict__ x,
                                               const int32_t *__restrict__ parent, const T *__restrict__ ec,
                                               T *__restrict__ xout, T omega) {
    // the static data (row, parents of the row's columns, inverse diagonal)
    // before the wait for the previous kernel when the row has eight slots
    const int i = bid_ * blockDim.x + threadIdx.x;
    const bool ok = i < nf, pre = ok && W == 8;
    T di = T(0), av8[8];
    int js8[8], pa8[8], pb8[8], pi0 = 0, pi1 = 0;
    if (ok) {
        di = dinv[i];
        pi0 = parent[2 * i];
        pi1 = parent[2 * i + 1];
    }
    if (pre) {
        const int4 c0 = *reinterpret_cast<const int4 *>(col + size_t(i) * 8);
        const int4 c1 = *reinterpret_cast<const int4 *>(col + size_t(i) * 8 + 4);
        js8[0] = c0.x; js8[1] = c0.y; js8[2] = c0.z; js8[3] = c0.w;
        js8[4] = c1.x; js8[5] = c1.y; js8[6] = c1.z; js8[7] = c1.w;
        load4(A + size_t(i) * 8, av8);
        load4(A + size_t(i) * 8 + 4, av8 + 4);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            pa8[q] = parent[2 * js8[q]];
            pb8[q] = parent[2 * js8[q] + 1];
        }
    }
    pdl_wait();
    if (!ok) return;
    T ax = T(0);
    if (pre) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int a = pa8[q], bb = pb8[q];
            const T pj = (a == bb) ? ec[a] : T(0.5) * (ec[a] + ec[bb]);
            ax = fma(av8[q], x[js8[q]] + pj, ax);
        }
        const T xi = x[i] + ((pi0 == pi1) ? ec[pi0] : T(0.5) * (ec[pi0] + ec[pi1]));
        xout[i] = fma(omega * di, b[i] - ax, xi);
        return;
    }
    const int32_t *c = col + size_t(i) * W;
    const T *arow = A + size_t(i) * W;
#pragma unroll 2
    for (int q = 0; q < W; q += 4) {
        const int4 cc = *reinterpret_cast<const int4 *>(c + q);
        T av[4];
        load4(arow + q, av);
        const int js[4] = {cc.x, cc.y, cc.z, cc.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = js[u], a = parent[2 * j], bb = parent[2 * j + 1];
            const T pj = (a == bb) ? ec[a] : T(0.5) * (ec[a] + ec[bb]);
            ax = fma(av[u], x[j] + pj, ax);
        }
    }
    const T xi = x[i] + ((pi0 == pi1) ? ec[pi0] : T(0.5) * (ec[pi0] + ec[pi1]));
    xout[i] = fma(omega * di, b[i] - ax, xi);
}
template <typename T>
__global__ void up_kernel(int nf, int W, const int32_t *__restrict__ col, const T *__restrict__ A,
                          const T *__restrict__ dinv, const T *__restrict__ b, const T *__restrict__ x,
                          const int32_t *__restrict__ parent, const T *__restrict__ ec, T *__restrict__ xout,
                          T omega) {
    up_kernel_impl<T>(blockIdx.x, gridDim.x, nf, W, col, A, dinv, b, x, parent, ec, xout, omega);
}
template <typename T>
struct up_kernel_args {
    int nb_;
    int nf;
    int W;
    const int32_t *col;
    const T *A;
    const T *dinv;
    const T *b;
    const T *x;
    const int32_t *parent;
    const T *ec;
    T *xout;
    T omega;
};
template <typename T>
__global__ void up_kernel_multi(const __grid_constant__ MultiP<up_kernel_args<T>> M) {
    int b_;
    const up_kernel_args<T> &q_ = M.a[merge_find(M.start, M.n, b_)];
    up_kernel_impl<T>(b_, q_.nb_, q_.nf, q_.W, q_.col, q_.A, q_.dinv, q_.b, q_.x, q_.parent, q_.ec, q_.xout,
        q_.omega);
}
template <typename T>
void up_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, int nf, int W, const int32_t *col,
                  const T *A, const T *dinv, const T *b, const T *x, const int32_t *parent, const T *ec, T *xout,
                  T omega) {
    if (Recorder *r_ = batch_recorder()) {
        up_kernel_args<T> q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.nf = nf;
        q_.W = W;
        q_.col = col;
        q_.A = A;
        q_.dinv = dinv;
        q_.b = b;
        q_.x = x;
        q_.parent = parent;
        q_.ec = ec;
        q_.xout = xout;
        q_.omega = omega;
        batch_record(r_, reinterpret_cast<const void *>(&up_kernel_multi<T>), q_, grid_, block_, smem_, kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &up_kernel<T>, grid_, block_, smem_, s_, nf, W, col, A, dinv, b, x, parent, ec, xout, omega);
}


// (A x)_i on a staged tail level: the row's W columns as 16-bit indices
// (row-major, one 16-byte load per eight), the values slot-major (slot q of
// row i at A[q * nv + i]), so that neither read has shared-memory bank
// conflicts across a warp of consecutive rows; the sum runs over the slots in
// order, as ell_row's does.
template <typename T>
__device__ __forceinline__ T tail_row(int i, int W, int nv, const uint16_t *__restrict__ col, const T *__restrict__ A,
                                      const T *__restrict__ x) {
    T ax = T(0);
    const uint16_t *c = col + size_t(i) * W;
    if (W == 8) {
        const uint4 cc = *reinterpret_cast<const uint4 *>(c);
        const uint32_t w[4] = {cc.x, cc.y, cc.z, cc.w};
#pragma unroll
        for (int q = 0; q < 8; ++q) ax = fma(A[q * nv + i], x[(w[q >> 1] >> (16 * (q & 1))) & 0xffffu], ax);
        return ax;
    }
    for (int q = 0; q < W; q += 4) {
        const uint2 cc = *reinterpret_cast<const uint2 *>(c + q);
        ax = fma(A[(q + 0) * nv + i], x[cc.x & 0xffffu], ax);
        ax = fma(A[(q + 1) * nv + i], x[cc.x >> 16], ax);
        ax = fma(A[(q + 2) * nv + i], x[cc.y & 0xffffu], ax);
        ax = fma(A[(q + 3) * nv + i], x[cc.y >> 16], ax);
    }
    return ax;
}

// x_j + (P e_c)_j: the midpoint prolongation of the coarse correction added on the fly
template <typename T>
__device__ __forceinline__ T prolonged(const int32_t *par, const T *x, const T *ec, int j) {
    const int p0 = par[2 * j], p1 = par[2 * j + 1];
    return x[j] + ((p0 == p1) ? ec[p0] : T(0.5) * (ec[p0] + ec[p1]));
}

// Fused steps over patches (HostPatches): one block per patch, one thread per
// patch row, the one-ring halo recomputed by every patch that needs it, so
// that a smoothing sweep and the step that consumes it share one launch.
// Every index a thread needs (its row's columns, local columns, the parents
// of its columns, its coarse vertex's children) is read from per-patch copies
// before the first barrier, and its row's operator values stay in registers:
// after the first phase only shared-memory gathers remain.  Every value is
// formed with the arithmetic of the unfused kernels (rows in ELL slot order).
__device__ __forceinline__ int4 load_cols(const int32_t *p) { return *reinterpret_cast<const int4 *>(p); }
__device__ __forceinline__ int cget(const int4 &c, int u) { return u == 0 ? c.x : u == 1 ? c.y : u == 2 ? c.z : c.w; }

// threads per patch block: FP32 rows fit 64 registers (1024 threads), FP64 rows 84 (768)
template <typename T>
constexpr int kPatchThreads = sizeof(T) == 4 ? 1024 : 768;
constexpr int kChildPrefetch = 8;     // children of a coarse vertex held in registers

// Going down one level, fused with the last pre-smoothing sweep.  Row s of
// patch F1: x' = x + omega D^-1 (b - A x) (x from global memory) into shared
// memory, and to xout for F0 rows (the pre-smoothed iterate; F0 sets of
// neighbouring patches overlap and write identical values); r = b - A x' on
// F0; b_c = R r for the patch's coarse vertices and, when xc is given, the
// coarse level's first sweep from zero, x_c = omega D_c^-1 b_c.
template <typename T, int WQ>
__device__ __forceinline__ void down_fused_kernel_impl(int bid_, int nb_, const int32_t *__restrict__ f_ptr,
                                                       const int32_t *__restrict__ f_n0,
                                                       const int32_t *__restrict__ f_ids,
                                                       const int32_t *__restrict__ f0_base,
                                                       const int32_t *__restrict__ lcol,
                                                       const int32_t *__restrict__ fcol,
                                                       const int32_t *__restrict__ c_ptr,
                                                       const int32_t *__restrict__ c_ids,
                                                       const int32_t *__restrict__ cc_ptr,
                                                       const int32_t *__restrict__ cc_slot,
                                                       const T *__restrict__ cc_w, const T *__restrict__ A,
                                                       const T *__restrict__ dinv, const T *__restrict__ b,
                                                       const T *__restrict__ x, T *__restrict__ xout,
                                                       const T *__restrict__ dinv_c, T omega, T *__restrict__ bc,
                                                       T *__restrict__ xc, int max_f1) {
    constexpr int W = 4 * WQ;
    extern __shared__ __align__(16) unsigned char patch_smem[];
    T *xs = reinterpret_cast<T *>(patch_smem);
    T *rs = xs + max_f1;
    const int blk = bid_, s = threadIdx.x;
    const int s0 = f_ptr[blk], n1 = f_ptr[blk + 1] - s0, n0 = f_n0[blk];
    const int c = c_ptr[blk] + s;
    const bool row = s < n1, row0 = s < n0, crow = c < c_ptr[blk + 1];
    int v = 0;
    int4 cols[WQ], lcs[WQ];
    if (row) {
        v = f_ids[s0 + s];
#pragma unroll
        for (int g = 0; g < WQ; ++g) cols[g] = load_cols(fcol + size_t(s0 + s) * W + 4 * g);
    }
    if (row0) {
        const int r0 = f0_base[blk];
#pragma unroll
        for (int g = 0; g < WQ; ++g) lcs[g] = load_cols(lcol + size_t(r0 + s) * W + 4 * g);
    }
    int cid = 0, k0 = 0, k1 = 0;
    int cs[kChildPrefetch];
    T cwv[kChildPrefetch];
    if (crow) {
        cid = c_ids[c];
        k0 = cc_ptr[c];
        k1 = cc_ptr[c + 1];
#pragma unroll
        for (int j = 0; j < kChildPrefetch; ++j) {
            cs[j] = k0 + j < k1 ? cc_slot[k0 + j] : 0;
            cwv[j] = k0 + j < k1 ? cc_w[k0 + j] : T(0);
        }
    }
    T av[W];
    T bv = T(0), dv = T(0);
    if (row) {
#pragma unroll
        for (int g = 0; g < WQ; ++g) load4(A + size_t(v) * W + 4 * g, av + 4 * g);
        dv = dinv[v];
    }
    // everything above is static (patch maps, operator rows): the vectors of
    // the previous kernel only from here on
    pdl_wait();
    if (row) {
        bv = b[v];
        T ax = T(0);
#pragma unroll
        for (int g = 0; g < WQ; ++g)
#pragma unroll
            for (int u = 0; u < 4; ++u) ax = fma(av[4 * g + u], x[cget(cols[g], u)], ax);
        const T xn = fma(omega * dv, bv - ax, x[v]);
        xs[s] = xn;
        if (row0) xout[v] = xn;
    }
    __syncthreads();
    if (row0) {
        T ax = T(0);
#pragma unroll
        for (int g = 0; g < WQ; ++g)
#pragma unroll
            for (int u = 0; u < 4; ++u) ax = fma(av[4 * g + u], xs[cget(lcs[g], u)], ax);
        rs[s] = bv - ax;
    }
    __syncthreads();
    if (crow) {
        T acc = T(0);
#pragma unroll
        for (int j = 0; j < kChildPrefetch; ++j)
            if (k0 + j < k1) acc = fma(cwv[j], rs[cs[j]], acc);
        for (int k = k0 + kChildPrefetch; k < k1; ++k) acc = fma(cc_w[k], rs[cc_slot[k]], acc);
        bc[cid] = acc;
        if (xc) xc[cid] = omega * dinv_c[cid] * acc;
    }
}
template <typename T, int WQ>
__global__ void __launch_bounds__(kPatchThreads<T>, 1) down_fused_kernel(const int32_t *__restrict__ f_ptr,
                                                                         const int32_t *__restrict__ f_n0,
                                                                         const int32_t *__restrict__ f_ids,
                                                                         const int32_t *__restrict__ f0_base,
                                                                         const int32_t *__restrict__ lcol,
                                                                         const int32_t *__restrict__ fcol,
                                                                         const int32_t *__restrict__ c_ptr,
                                                                         const int32_t *__restrict__ c_ids,
                                                                         const int32_t *__restrict__ cc_ptr,
                                                                         const int32_t *__restrict__ cc_slot,
                                                                         const T *__restrict__ cc_w,
                                                                         const T *__restrict__ A,
                                                                         const T *__restrict__ dinv,
                                                                         const T *__restrict__ b,
                                                                         const T *__restrict__ x,
                                                                         T *__restrict__ xout,
                                                                         const T *__restrict__ dinv_c, T omega,
                                                                         T *__restrict__ bc, T *__restrict__ xc,
                                                                         int max_f1) {
    down_fused_kernel_impl<T, WQ>(blockIdx.x, gridDim.x, f_ptr, f_n0, f_ids, f0_base, lcol, fcol, c_ptr, c_ids,
        cc_ptr, cc_slot, cc_w, A, dinv, b, x, xout, dinv_c, omega, bc, xc, max_f1);
}
template <typename T, int WQ>
struct down_fused_kernel_args {
    int nb_;
    const int32_t *f_ptr;
    const int32_t *f_n0;
    const int32_t *f_ids;
    const int32_t *f0_base;
    const int32_t *lcol;
    const int32_t *fcol;
    const int32_t *c_ptr;
    const int32_t *c_ids;
    const int32_t *cc_ptr;
    const int32_t *cc_slot;
    const T *cc_w;
    const T *A;
    const T *dinv;
    const T *b;
    const T *x;
    T *xout;
    const T *dinv_c;
    T omega;
    T *bc;
    T *xc;
    int max_f1;
};
template <typename T, int WQ>
__global__ void __launch_bounds__(kPatchThreads<T>, 1) down_fused_kernel_multi(const __grid_constant__ MultiP<down_fused_kernel_args<T, WQ>> M) {
    int b_;
    const down_fused_kernel_args<T, WQ> &q_ = M.a[merge_find(M.start, M.n, b_)];
    down_fused_kernel_impl<T, WQ>(b_, q_.nb_, q_.f_ptr, q_.f_n0, q_.f_ids, q_.f0_base, q_.lcol, q_.fcol, q_.c_ptr,
        q_.c_ids, q_.cc_ptr, q_.cc_slot, q_.cc_w, q_.A, q_.dinv, q_.b, q_.x, q_.xout, q_.dinv_c, q_.omega, q_.bc,
        q_.xc, q_.max_f1);
}
template <typename T, int WQ>
void down_fused_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, const int32_t *f_ptr,
                          const int32_t *f_n0, const int32_t *f_ids, const int32_t *f0_base, const int32_t *lcol,
                          const int32_t *fcol, const int32_t *c_ptr, const int32_t *c_ids, const int32_t *cc_ptr,
                          const int32_t *cc_slot, const T *cc_w, const T *A, const T *dinv, const T *b, const T *x,
                          T *xout, const T *dinv_c, T omega, T *bc, T *xc, int max_f1) {
    if (Recorder *r_ = batch_recorder()) {
        down_fused_kernel_args<T, WQ> q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.f_ptr = f_ptr;
        q_.f_n0 = f_n0;
        q_.f_ids = f_ids;
        q_.f0_base = f0_base;
        q_.lcol = lcol;
        q_.fcol = fcol;
        q_.c_ptr = c_ptr;
        q_.c_ids = c_ids;
        q_.cc_ptr = cc_ptr;
        q_.cc_slot = cc_slot;
        q_.cc_w = cc_w;
        q_.A = A;
        q_.dinv = dinv;
        q_.b = b;
        q_.x = x;
        q_.xout = xout;
        q_.dinv_c = dinv_c;
        q_.omega = omega;
        q_.bc = bc;
        q_.xc = xc;
        q_.max_f1 = max_f1;
        batch_record(r_, reinterpret_cast<const void *>(&down_fused_kernel_multi<T, WQ>), q_, grid_, block_, smem_, kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &down_fused_kernel<T, WQ>, grid_, block_, smem_, s_, f_ptr, f_n0, f_ids, f0_base, lcol, fcol, c_ptr, c_ids,
        cc_ptr, cc_slot, cc_w, A, dinv, b, x, xout, dinv_c, omega, bc, xc, max_f1);
}


// (P e_c) at a vertex with parents (pa, pb): the midpoint prolongation
template <typename T>
__device__ __forceinline__ T prolong_at(const T *__restrict__ ec, int pa, int pb) {
    return (pa == pb) ? ec[pa] : T(0.5) * (ec[pa] + ec[pb]);
}

// Going up one level, fused with the second post-smoothing sweep.  Row s of
// the patch (owned vertices, then their neighbours): x' = (x + P e_c) +
// omega D^-1 (b - A (x + P e_c)) into shared memory (the prolongation formed
// on the fly, as up_kernel does); then x'' = x' + omega D^-1 (b - A x') on the
// owned rows to xout.
template <typename T, int WQ>
__device__ __forceinline__ void up_fused_kernel_impl(int bid_, int nb_, const int32_t *__restrict__ g_ptr,
                                                     const int32_t *__restrict__ g_nown,
                                                     const int32_t *__restrict__ g_ids,
                                                     const int32_t *__restrict__ g0_base,
                                                     const int32_t *__restrict__ glcol,
                                                     const int32_t *__restrict__ gcol,
                                                     const int32_t *__restrict__ gpar,
                                                     const int32_t *__restrict__ grow_par, const T *__restrict__ A,
                                                     const T *__restrict__ dinv, const T *__restrict__ b,
                                                     const T *__restrict__ x, const T *__restrict__ ec,
                                                     T *__restrict__ xout, T omega) {
    constexpr int W = 4 * WQ;
    extern __shared__ __align__(16) unsigned char patch_smem[];
    T *xs = reinterpret_cast<T *>(patch_smem);
    const int blk = bid_, s = threadIdx.x;
    const int s0 = g_ptr[blk], n1 = g_ptr[blk + 1] - s0, nown = g_nown[blk];
    const bool row = s < n1, own = s < nown;
    int v = 0;
    int4 cols[WQ], lcs[WQ], par[2 * WQ];
    int2 rp = make_int2(0, 0);
    if (row) {
        v = g_ids[s0 + s];
#pragma unroll
        for (int g = 0; g < WQ; ++g) cols[g] = load_cols(gcol + size_t(s0 + s) * W + 4 * g);
#pragma unroll
        for (int g = 0; g < 2 * WQ; ++g) par[g] = load_cols(gpar + size_t(s0 + s) * 2 * W + 4 * g);
        rp = *reinterpret_cast<const int2 *>(grow_par + 2 * size_t(s0 + s));
    }
    if (own) {
        const int r0 = g0_base[blk];
#pragma unroll
        for (int g = 0; g < WQ; ++g) lcs[g] = load_cols(glcol + size_t(r0 + s) * W + 4 * g);
    }
    T av[W];
    T bv = T(0), wv = T(0), x3 = T(0);
    if (row) {
#pragma unroll
        for (int g = 0; g < WQ; ++g) load4(A + size_t(v) * W + 4 * g, av + 4 * g);
        wv = omega * dinv[v];
    }
    // everything above is static (patch maps, operator rows): the vectors of
    // the previous kernels only from here on
    pdl_wait();
    if (row) {
        bv = b[v];
        T ax = T(0);
#pragma unroll
        for (int g = 0; g < WQ; ++g)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int q = 4 * g + u;
                const int4 pq = par[q / 2];
                const int pa = (q & 1) ? pq.z : pq.x, pb = (q & 1) ? pq.w : pq.y;
                ax = fma(av[q], x[cget(cols[g], u)] + prolong_at(ec, pa, pb), ax);
            }
        x3 = fma(wv, bv - ax, x[v] + prolong_at(ec, rp.x, rp.y));
        xs[s] = x3;
    }
    __syncthreads();
    if (own) {
        T ax = T(0);
#pragma unroll
        for (int g = 0; g < WQ; ++g)
#pragma unroll
            for (int u = 0; u < 4; ++u) ax = fma(av[4 * g + u], xs[cget(lcs[g], u)], ax);
        xout[v] = fma(wv, bv - ax, x3);
    }
}
template <typename T, int WQ>
__global__ void __launch_bounds__(kPatchThreads<T>, 1) up_fused_kernel(const int32_t *__restrict__ g_ptr,
                                                                       const int32_t *__restrict__ g_nown,
                                                                       const int32_t *__restrict__ g_ids,
                                                                       const int32_t *__restrict__ g0_base,
                                                                       const int32_t *__restrict__ glcol,
                                                                       const int32_t *__restrict__ gcol,
                                                                       const int32_t *__restrict__ gpar,
                                                                       const int32_t *__restrict__ grow_par,
                                                                       const T *__restrict__ A,
                                                                       const T *__restrict__ dinv,
                                                                       const T *__restrict__ b,
                                                                       const T *__restrict__ x,
                                                                       const T *__restrict__ ec, T *__restrict__ xout,
                                                                       T omega) {
    up_fused_kernel_impl<T, WQ>(blockIdx.x, gridDim.x, g_ptr, g_nown, g_ids, g0_base, glcol, gcol, gpar, grow_par, A,
        dinv, b, x, ec, xout, omega);
}
template <typename T, int WQ>
struct up_fused_kernel_args {
    int nb_;
    const int32_t *g_ptr;
    const int32_t *g_nown;
    const int32_t *g_ids;
    const int32_t *g0_base;
    const int32_t *glcol;
    const int32_t *gcol;
    const int32_t *gpar;
    const int32_t *grow_par;
    const T *A;
    const T *dinv;
    const T *b;
    const T *x;
    const T *ec;
    T *xout;
    T omega;
};
template <typename T, int WQ>
__global__ void __launch_bounds__(kPatchThreads<T>, 1) up_fused_kernel_multi(const __grid_constant__ MultiP<up_fused_kernel_args<T, WQ>> M) {
    int b_;
    const up_fused_kernel_args<T, WQ> &q_ = M.a[merge_find(M.start, M.n, b_)];
    up_fused_kernel_impl<T, WQ>(b_, q_.nb_, q_.g_ptr, q_.g_nown, q_.g_ids, q_.g0_base, q_.glcol, q_.gcol, q_.gpar,
        q_.grow_par, q_.A, q_.dinv, q_.b, q_.x, q_.ec, q_.xout, q_.omega);
}
template <typename T, int WQ>
void up_fused_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, const int32_t *g_ptr,
                        const int32_t *g_nown, const int32_t *g_ids, const int32_t *g0_base, const int32_t *glcol,
                        const int32_t *gcol, const int32_t *gpar, const int32_t *grow_par, const T *A, const T *dinv,
                        const T *b, const T *x, const T *ec, T *xout, T omega) {
    if (Recorder *r_ = batch_recorder()) {
        up_fused_kernel_args<T, WQ> q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.g_ptr = g_ptr;
        q_.g_nown = g_nown;
        q_.g_ids = g_ids;
        q_.g0_base = g0_base;
        q_.glcol = glcol;
        q_.gcol = gcol;
        q_.gpar = gpar;
        q_.grow_par = grow_par;
        q_.A = A;
        q_.dinv = dinv;
        q_.b = b;
        q_.x = x;
        q_.ec = ec;
        q_.xout = xout;
        q_.omega = omega;
        batch_record(r_, reinterpret_cast<const void *>(&up_fused_kernel_multi<T, WQ>), q_, grid_, block_, smem_, kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &up_fused_kernel<T, WQ>, grid_, block_, smem_, s_, g_ptr, g_nown, g_ids, g0_base, glcol, gcol, gpar, grow_par,
        A, dinv, b, x, ec, xout, omega);
}


// The V-cycle over the small levels in one CTA.  The levels' operators
// (ELL values and columns, inverse diagonals), transfer lists and, when it
// fits, the coarsest level's FP64 inverse were packed at condensation into one
// image laid out exactly as this kernel's shared memory, headed by a table of
// sizes and offsets; a few bulk copies (cp.async.bulk, one mbarrier with a
// transaction count) stage it, then the steps run with __syncthreads between
// them.  Level 0 of the tail takes b from global memory and returns x there;
// the last level is solved with its dense inverse.  The image and every
// chunk of it start 16-byte aligned.
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

// bounded wait on phase 0 of the barrier; false if the limit ran out
__device__ __forceinline__ bool bar_wait(uint64_t *bar, long long limit) {
    for (long long it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(smem_u32(bar)) : "memory");
        if (done) return true;
    }
    return false;
}

// dense FP64 product x = inv b of the coarsest level (n rows): four lanes per
// row (FP64 arithmetic is a narrow pipe: few adds in the tree), each summing
// every fourth column, combined by a fixed two-step shuffle.  Whole warps take
// part in every shuffle: the row loop runs to a multiple of 8.
template <typename T>
__device__ __forceinline__ void coarse_product(const double *inv, int n, const T *b, T *x) {
    const int sub = threadIdx.x & 3, ng = blockDim.x >> 2;
    for (int i = threadIdx.x >> 2; i < ((n + 7) & ~7); i += ng) {
        double acc = 0.0;
        if (i < n)
            for (int j = sub; j < n; j += 4) acc = fma(inv[size_t(i) * n + j], double(b[j]), acc);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        if (i < n && sub == 0) x[i] = T(acc);
    }
}


// x = inv b on a coarsest level too large for the single-CTA cycle (FP64
// inverse, FP64 sums in every precision): one block of four warps per row,
// each thread summing pairs of columns 256 apart (16-byte loads, all of a
// thread's loads independent), then a fixed shuffle tree per warp and the
// four warp sums in order.
template <typename T>
__device__ __forceinline__ void coarse_dense_kernel_impl(int bid_, int nb_, const double *__restrict__ inv, int n,
                                                         const T *__restrict__ b, T *__restrict__ x) {
    __shared__ double part[4];
    const int row = bid_, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double *a = inv + size_t(row) * n;
    double acc = 0.0;
    if ((n & 1) == 0) {
        // rows start on 16-byte boundaries when n is even
#pragma unroll 4
        for (int j = 2 * tid; j < n; j += 256) {
            const double2 av = *reinterpret_cast<const double2 *>(a + j);
            acc = fma(av.x, double(b[j]), acc);
            acc = fma(av.y, double(b[j + 1]), acc);
        }
    } else {
#pragma unroll 4
        for (int j = tid; j < n; j += 128) acc = fma(a[j], double(b[j]), acc);
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) part[warp] = acc;
    __syncthreads();
    if (tid == 0) x[row] = T(((part[0] + part[1]) + part[2]) + part[3]);
    (void)nb_;
}
template <typename T>
__global__ void __launch_bounds__(128) coarse_dense_kernel(const double *inv, int n, const T *b, T *x) {
    pdl_wait();
    coarse_dense_kernel_impl<T>(blockIdx.x, gridDim.x, inv, n, b, x);
}
template <typename T>
struct coarse_dense_kernel_args {
    int nb_;
    const double *inv;
    int n;
    const T *b;
    T *x;
};
template <typename T>
__global__ void __launch_bounds__(128) coarse_dense_kernel_multi(const __grid_constant__ MultiP<coarse_dense_kernel_args<T>> M) {
    pdl_wait();
    int b_;
    const coarse_dense_kernel_args<T> &q_ = M.a[merge_find(M.start, M.n, b_)];
    coarse_dense_kernel_impl<T>(b_, q_.nb_, q_.inv, q_.n, q_.b, q_.x);
}
template <typename T>
void coarse_dense_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, const double *inv, int n,
                            const T *b, T *x) {
    if (Recorder *r_ = batch_recorder()) {
        coarse_dense_kernel_args<T> q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.inv = inv;
        q_.n = n;
        q_.b = b;
        q_.x = x;
        batch_record(r_, reinterpret_cast<const void *>(&coarse_dense_kernel_multi<T>), q_, grid_, block_, smem_, kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &coarse_dense_kernel<T>, grid_, block_, smem_, s_, inv, n, b, x);
}

// Every array pointer below is the shared-memory base plus an offset from the
// level table, so that the compiler addresses shared memory directly.
template <typename T>
__device__ __forceinline__ void tail_kernel_impl(int bid_, int nb_, TailArgs a) {
    extern __shared__ __align__(16) unsigned char tail_smem[];
    __shared__ __align__(8) uint64_t bar;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // the image (level table, operators, transfers, inverse) in chunks of at
    // most 64 KB, one per lane of warp 0, after lane 0 has set the byte count
    if (tid < 32) {
        if (tid == 0)
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                         :: "r"(smem_u32(&bar)), "r"(a.img_bytes) : "memory");
        __syncwarp();
        constexpr uint32_t kChunk = 64 * 1024;
        const uint32_t o = uint32_t(tid) * kChunk;
        if (o < a.img_bytes) bulk_g2s(tail_smem + o, a.img + o, min(kChunk, a.img_bytes - o), &bar);
    }
    // the image is static: its copies are issued before the wait for the
    // previous kernel, whose output (the first level's right-hand side) is read
    // only after it
    pdl_wait();
    const T om = T(a.omega);
    auto PT = [&](int32_t o) { return reinterpret_cast<T *>(tail_smem + o); };
    auto PI = [&](int32_t o) { return reinterpret_cast<int32_t *>(tail_smem + o); };
    // meanwhile, with plain loads into the scratch space after the image: the
    // first level's right-hand side and its first pre-smoothing sweep from
    // zero, x = omega D^-1 b (the inverse diagonal read from global memory)
    {
        const T *btop = static_cast<const T *>(a.b_top);
        const T *d0 = static_cast<const T *>(a.dinv0);
        T *b0 = PT(a.ob0), *x0 = PT(a.ox0);
        for (int i = tid; i < a.nv0; i += nt) {
            const T bi = btop[i];
            b0[i] = bi;
            x0[i] = a.nu1 == 0 ? T(0) : om * d0[i] * bi;
        }
    }
    if (!bar_wait(&bar, 1ll << 22)) {
        // the copies did not complete: record it, give them one more bounded
        // wait so none is left writing into this CTA's shared memory, return
        if (tid == 0) atomicOr(a.status, 8);
        bar_wait(&bar, 1ll << 22);
        return;
    }
    __syncthreads();
    TailHdr *H = reinterpret_cast<TailHdr *>(tail_smem);   // staged level table (ox/ox2 rewritten below)
    const int last = a.nlev - 1;
    // ---- down: x holds the first sweep (or zero) on entry to each level
    for (int l = 0; l < last; ++l) {
        const TailHdr h = H[l], hc = H[l + 1];
        const int nv = h.nv, W = h.W;
        const uint16_t *cl = reinterpret_cast<const uint16_t *>(tail_smem + h.ocol);
        const T *A = PT(h.oA), *D = PT(h.oD), *b = PT(h.ob);
        T *r = PT(h.orr);
        int32_t ox = h.ox, ox2 = h.ox2;
        for (int k = 1; k < a.nu1; ++k) {
            const T *x = PT(ox);
            T *x2 = PT(ox2);
            for (int i = tid; i < nv; i += nt) x2[i] = fma(om * D[i], b[i] - tail_row(i, W, nv, cl, A, x), x[i]);
            __syncthreads();
            const int32_t t = ox; ox = ox2; ox2 = t;
        }
        {
            const T *x = PT(ox);
            for (int i = tid; i < nv; i += nt) r[i] = b[i] - tail_row(i, W, nv, cl, A, x);
        }
        if (tid == 0) { H[l].ox = ox; H[l].ox2 = ox2; }   // read again only after later barriers
        __syncthreads();
        // restriction, with the coarse level's first sweep from zero
        const int32_t *cp = PI(hc.ocp), *ci = PI(hc.oci);
        const T *cw = PT(hc.ocw), *Dc = PT(hc.oD);
        T *bc = PT(hc.ob), *xc = PT(hc.ox);
        const bool smooth_c = l + 1 < last;
        for (int i = tid; i < hc.nv; i += nt) {
            T acc = T(0);
            for (int k = cp[i]; k < cp[i + 1]; ++k) acc = fma(cw[k], r[ci[k]], acc);
            bc[i] = acc;
            if (smooth_c) xc[i] = a.nu1 == 0 ? T(0) : om * Dc[i] * acc;
        }
        __syncthreads();
    }
    // ---- coarsest: dense FP64 inverse, FP64 sums in every precision
    {
        const TailHdr h = H[last];
        if (a.inv_off >= 0) coarse_product<T>(reinterpret_cast<const double *>(tail_smem + a.inv_off), h.nv, PT(h.ob), PT(h.ox));
        else coarse_product<T>(a.inv, h.nv, PT(h.ob), PT(h.ox));
        __syncthreads();
    }
    // ---- up: x += P e_c in place (a separate step: forming it on the fly in
    // the sweep multiplies the shared-memory gathers), then post-smoothing
    int32_t oec = H[last].ox;
    for (int l = last - 1; l >= 0; --l) {
        const TailHdr h = H[l];
        const int nv = h.nv, W = h.W;
        const uint16_t *cl = reinterpret_cast<const uint16_t *>(tail_smem + h.ocol);
        const int32_t *par = PI(H[l + 1].opar);
        const T *A = PT(h.oA), *D = PT(h.oD), *b = PT(h.ob);
        int32_t ox = h.ox, ox2 = h.ox2;
        {
            const T *ec = PT(oec);
            T *x = PT(ox);
            for (int i = tid; i < nv; i += nt) x[i] = prolonged(par, x, ec, i);
        }
        __syncthreads();
        for (int k = 0; k < a.nu2; ++k) {
            const T *x = PT(ox);
            T *x2 = PT(ox2);
            for (int i = tid; i < nv; i += nt) x2[i] = fma(om * D[i], b[i] - tail_row(i, W, nv, cl, A, x), x[i]);
            __syncthreads();
            const int32_t t = ox; ox = ox2; ox2 = t;
        }
        oec = ox;
    }
    T *xtop = static_cast<T *>(a.x_top);
    const T *ec = PT(oec);
    for (int i = tid; i < a.nv0; i += nt) xtop[i] = ec[i];
}
template <typename T>
__global__ void __launch_bounds__(1024, 1) tail_kernel(TailArgs a) {
    tail_kernel_impl<T>(blockIdx.x, gridDim.x, a);
}
template <typename T>
struct tail_kernel_args {
    int nb_;
    TailArgs a;
};
template <typename T>
__global__ void __launch_bounds__(1024, 1) tail_kernel_multi(const __grid_constant__ MultiP<tail_kernel_args<T>> M) {
    int b_;
    const tail_kernel_args<T> &q_ = M.a[merge_find(M.start, M.n, b_)];
    tail_kernel_impl<T>(b_, q_.nb_, q_.a);
}
template <typename T>
void tail_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, TailArgs a) {
    if (Recorder *r_ = batch_recorder()) {
        tail_kernel_args<T> q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.a = a;
        batch_record(r_, reinterpret_cast<const void *>(&tail_kernel_multi<T>), q_, grid_, block_, smem_, kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &tail_kernel<T>, grid_, block_, smem_, s_, a);
}


}  // namespace

template <typename T>
cudaError_t launch_p1_jacobi(const DevLevel &L, const T *A, const T *dinv, const T *b, const T *x, T *xout, T omega,
                             bool first, cudaStream_t s) {
    jacobi_kernel_go<T>(blocks(L.nv, 256), 256, 0, s, L.nv, L.width, L.col, A, dinv, b, x, xout, omega, first ? 1 : 0);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_p1_prolong_add(const DevLevel &coarse, int nv_fine, const T *ec, T *xf, cudaStream_t s) {
    prolong_add_kernel_go<T>(blocks(nv_fine, 256), 256, 0, s, nv_fine, coarse.parent, ec, xf);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_p1_down(const DevLevel &fine, const DevLevel &coarse, const T *A_f, const T *b_f, const T *x_f,
                           const T *dinv_c, T omega, T *b_c, T *x_c, cudaStream_t s) {
    const T *cw = sizeof(T) == 4 ? reinterpret_cast<const T *>(coarse.child_w32) : reinterpret_cast<const T *>(coarse.child_w);
    down_kernel_go<T>(blocks(size_t(coarse.nv) * 8, 256), 256, 0, s, coarse.nv, coarse.child_ptr, coarse.child_idx, cw,
                                                                      fine.nv, fine.width, fine.col, A_f, b_f, x_f, dinv_c,
                                                                      omega, b_c, x_c);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_p1_up(const DevLevel &fine, const DevLevel &coarse, const T *A_f, const T *dinv_f, const T *b_f,
                         const T *x_f, const T *ec, T *xout, T omega, cudaStream_t s) {
    up_kernel_go<T>(blocks(fine.nv, 256), 256, 0, s, fine.nv, fine.width, fine.col, A_f, dinv_f, b_f, x_f,
                                                      coarse.parent, ec, xout, omega);
    return cudaGetLastError();
}
// The patch kernels run one thread per row of the largest patch and hold a
// row's operator values in registers: ELL widths 4 and 8.
template <typename T>
bool p1_patch_ok(const DevLevel &L) {
    return L.nb > 0 && (L.width == 4 || L.width == 8) && L.max_f1 <= kPatchThreads<T> &&
           L.max_g1 <= kPatchThreads<T> && sizeof(T) * size_t(L.max_f1 + L.max_f0) <= 48 * 1024;
}
inline unsigned patch_threads(int rows) { return unsigned(std::max(64, (rows + 31) / 32 * 32)); }

template <typename T>
cudaError_t launch_p1_down_fused(const DevLevel &fine, const DevLevel &coarse, const T *A_f, const T *dinv_f,
                                 const T *b_f, const T *x_f, T *xout_f, const T *dinv_c, T omega, T *b_c, T *x_c,
                                 cudaStream_t s) {
    if (!p1_patch_ok<T>(fine)) return cudaErrorInvalidValue;
    const T *ccw = sizeof(T) == 4 ? reinterpret_cast<const T *>(fine.pcc_w32) : reinterpret_cast<const T *>(fine.pcc_w);
    const size_t smem = sizeof(T) * size_t(fine.max_f1 + fine.max_f0);
    auto k = fine.width == 4 ? down_fused_kernel_go<T, 1> : down_fused_kernel_go<T, 2>;
    k(fine.nb, patch_threads(fine.max_f1), smem, s, fine.pf_ptr, fine.pf_n0, fine.pf_ids, fine.pf0_base, fine.plcol,
      fine.pfcol, fine.pc_ptr, fine.pc_ids, fine.pcc_ptr, fine.pcc_slot, ccw, A_f, dinv_f, b_f, x_f, xout_f, dinv_c,
      omega, b_c, x_c, fine.max_f1);
    (void)coarse;
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_p1_up_fused(const DevLevel &fine, const DevLevel &coarse, const T *A_f, const T *dinv_f,
                               const T *b_f, const T *x_f, const T *ec, T *xout, T omega, cudaStream_t s) {
    if (!p1_patch_ok<T>(fine)) return cudaErrorInvalidValue;
    const size_t smem = sizeof(T) * size_t(fine.max_g1);
    auto k = fine.width == 4 ? up_fused_kernel_go<T, 1> : up_fused_kernel_go<T, 2>;
    k(fine.nb, patch_threads(fine.max_g1), smem, s, fine.pg_ptr, fine.pg_nown, fine.pg_ids, fine.pg0_base,
      fine.pglcol, fine.pgcol, fine.pgpar, fine.pgrow_par, A_f, dinv_f, b_f, x_f, ec, xout, omega);
    (void)coarse;
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_p1_coarse_dense(const double *inv, int n, const T *b, T *x, cudaStream_t s) {
    coarse_dense_kernel_go<T>(unsigned(n), 128, 0, s, inv, n, b, x);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_p1_tail(const TailArgs &a, size_t smem, cudaStream_t s) {
    // one fixed limit for every handle: the attribute is process-wide, so a
    // per-handle value could be lowered by another thread between set and launch
    if (smem > kTailSmemMax) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(tail_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kTailSmemMax));
    if (e != cudaSuccess) return e;
    tail_kernel_go<T>(1, 1024, smem, s, a);
    return cudaGetLastError();
}

namespace {

// one tail level's ELL arrays in the staged layout (see tail_row)
template <typename T>
__global__ void tail_pack_kernel(const int32_t *__restrict__ col, const T *__restrict__ A, int nv, int W,
                                 uint16_t *__restrict__ col16, T *__restrict__ At) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nv * W) return;
    const int i = k / W, q = k % W;
    col16[k] = static_cast<uint16_t>(col[k]);
    At[size_t(q) * nv + i] = A[k];
}

}  // namespace

cudaError_t launch_tail_pack(const int32_t *col, const void *A, size_t tsz, int nv, int W, void *col_dst, void *A_dst,
                             cudaStream_t s) {
    if (nv > 65536 || W % 4 != 0) return cudaErrorInvalidValue;
    const unsigned nb = unsigned((size_t(nv) * W + 255) / 256);
    if (nb == 0) return cudaSuccess;
    if (tsz == sizeof(double))
        tail_pack_kernel<double><<<nb, 256, 0, s>>>(col, static_cast<const double *>(A), nv, W,
                                                    static_cast<uint16_t *>(col_dst), static_cast<double *>(A_dst));
    else
        tail_pack_kernel<float><<<nb, 256, 0, s>>>(col, static_cast<const float *>(A), nv, W,
                                                   static_cast<uint16_t *>(col_dst), static_cast<float *>(A_dst));
    return cudaGetLastError();
}

#define HDG_P1_INST(T)                                                                                         \
    template cudaError_t launch_p1_jacobi<T>(const DevLevel &, const T *, const T *, const T *, const T *, T *, \
                                             T, bool, cudaStream_t);                                           \
    template cudaError_t launch_p1_prolong_add<T>(const DevLevel &, int, const T *, T *, cudaStream_t);         \
    template cudaError_t launch_p1_down<T>(const DevLevel &, const DevLevel &, const T *, const T *, const T *,  \
                                           const T *, T, T *, T *, cudaStream_t);                               \
    template cudaError_t launch_p1_up<T>(const DevLevel &, const DevLevel &, const T *, const T *, const T *,    \
                                         const T *, const T *, T *, T, cudaStream_t);                           \
    template cudaError_t launch_p1_down_fused<T>(const DevLevel &, const DevLevel &, const T *, const T *,        \
                                                 const T *, const T *, T *, const T *, T, T *, T *, cudaStream_t); \
    template cudaError_t launch_p1_up_fused<T>(const DevLevel &, const DevLevel &, const T *, const T *, const T *, \
                                               const T *, const T *, T *, T, cudaStream_t);                        \
    template bool p1_patch_ok<T>(const DevLevel &);                                                          \
    template cudaError_t launch_p1_tail<T>(const TailArgs &, size_t, cudaStream_t);                           \
    template cudaError_t launch_p1_coarse_dense<T>(const double *, int, const T *, T *, cudaStream_t);
HDG_P1_INST(double)
HDG_P1_INST(float)

}  // namespace hdg
