// Two-float arithmetic for the FP64 steps of the mixed-precision path: the
// condensed right-hand side (step 1 of the Schur-complement solve, Sec. 3.3),
// the refinement residual g - S lambda (Eq. schur_system) and the recovery of
// the cell unknowns (step 3).  GB300's FP64 pipe is far slower than its FP32
// one, and these steps are FP64-FMA bound there, not HBM bound.
//
// Every stored FP64 matrix entry a is kept as a pair (hi, lo) = (rn(a),
// rn(a - hi)) of floats (8 bytes, like the double), every FP64 input is split
// the same way once per use, and a sum of products is carried as
//   s + c:  s the running sum of the rounded leading products hi_a*hi_x, added
//           by error-free TwoSum steps; c the float sum of the exact product
//           errors (by FMA), the cross terms hi_a*lo_x + lo_a*hi_x and the
//           TwoSum errors.
// The dropped lo_a*lo_x and the rounding of c leave a relative error of about
// n * 2^-48 of sum |a_i x_i| (FP64: n * 2^-53), at a dozen FP32 operations per
// term.  Values must lie in the FP32 range (|v| < 3e38); an overflow shows up
// as Inf/NaN in the refinement residual, which the solver reports.
#include "common.h"

namespace hdg {

// launch family of this file for pdl_launch (facet-row kernels); the kernel
// that ends an inner solve goes with the Krylov kernels
constexpr unsigned kPdlFamily = 1;
constexpr unsigned kPdlKrylov = 4;

namespace {

inline unsigned blocks(size_t n, int bs) { return unsigned((n + bs - 1) / bs); }

// The cell kernels take 32 consecutive cells per block (lane = cell): the
// cells' right-hand sides r_K = (r_u, r_h) are read as contiguous chunks,
// split once into shared memory and shared by the warps, which take the output
// rows in turn; per-cell matrices, split into pairs of row entries
// ([row][col pair][N], split_pairs_kernel), load coalesced, 16 bytes per lane.
constexpr int kCells = kFFCells;
constexpr int kCellsPad = kCells + 1;

__global__ void split_kernel(const double *__restrict__ a, float2 *__restrict__ out, size_t n) {
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) out[i] = split(a[i]);
}

// A per-cell matrix a[(row * cols + col) * N + K] split into pairs of
// consecutive row entries, in tiles of kCells cells: the pair (col 2cp, col
// 2cp + 1, or zeros past the row's end) of plane pc = row * CP + cp, CP =
// (cols + 1) / 2, for cell K sits at out[((K / kCells) * rows * CP + pc) *
// kCells + K % kCells].  One 16-byte load per lane brings two entries of a row,
// a warp's loads are coalesced, and a block of kCells cells streams one
// contiguous tile.
__global__ void split_pairs_kernel(const double *__restrict__ a, float4 *__restrict__ out, int rows, int cols,
                                   size_t N) {
    const int CP = (cols + 1) / 2;
    const size_t np = size_t(rows) * CP;
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= np * N) return;
    const size_t K = i % N, pc = i / N;
    const int row = int(pc / CP), c0 = 2 * int(pc % CP);
    const float2 lo = split(a[(size_t(row) * cols + c0) * N + K]);
    const float2 hi = c0 + 1 < cols ? split(a[(size_t(row) * cols + c0 + 1) * N + K]) : make_float2(0.f, 0.f);
    out[ff_pair_index(K, pc, np)] = make_float4(lo.x, lo.y, hi.x, hi.y);
}

// acc += sum over the NCOL entries of one row (pairs p[cp * kCells], cp <
// (NCOL + 1) / 2, within the cell's tile) times x[col][lane], in column order
template <int NCOL>
__device__ __forceinline__ void row_pairs(FFAcc &acc, const float4 *__restrict__ p, const float2 (*x)[kCellsPad],
                                          int lane, bool negate = false) {
    constexpr int CP = (NCOL + 1) / 2;
#pragma unroll 3
    for (int cp = 0; cp < CP; ++cp) {
        const float4 v = __ldg(p + size_t(cp) * kCells);
        const float2 a0 = negate ? make_float2(-v.x, -v.y) : make_float2(v.x, v.y);
        acc.add(a0, x[2 * cp][lane]);
        if (2 * cp + 1 < NCOL) {
            const float2 a1 = negate ? make_float2(-v.z, -v.w) : make_float2(v.z, v.w);
            acc.add(a1, x[2 * cp + 1][lane]);
        }
    }
}

// The refinement iterate lambda is kept only as float pairs (hi, lo), the form
// the residual kernel reads; the correction x += scale * d then runs on the
// FP32 pipe, and the pairs are joined into FP64 once, when the solve ends.
// (hi, lo) += (sh + sl) * d, (sh, sl) = split(scale) formed once per block:
// the leading product by FMA with its exact error, the cross term sl * d, a
// TwoSum of the leading parts, the trailing parts added to its error and a
// renormalisation (about 2^-46 relative).  first: the iterate is zero and not
// read.
__device__ __forceinline__ float2 ff_add_scaled(float2 xv, float2 sc, float di, bool first) {
    const float ph = __fmul_rn(sc.x, di);
    const float pl = __fmaf_rn(sc.y, di, __fmaf_rn(sc.x, di, -ph));
    if (first) {
        const float t = __fadd_rn(ph, pl);
        return make_float2(t, __fsub_rn(pl, __fsub_rn(t, ph)));
    }
    const float t = __fadd_rn(xv.x, ph);
    const float bp = __fsub_rn(t, xv.x);
    float e = __fadd_rn(__fsub_rn(xv.x, __fsub_rn(t, bp)), __fsub_rn(ph, bp));
    e = __fadd_rn(e, __fadd_rn(xv.y, pl));
    const float hi = __fadd_rn(t, e);
    return make_float2(hi, __fsub_rn(e, __fsub_rn(hi, t)));
}
__device__ __forceinline__ void ff_axpy_kernel_impl(int bid_, int nb_, float2 *__restrict__ x2,
                                                    const float *__restrict__ d, const double *__restrict__ scale,
                                                    size_t n, int first) {
    // the entry's loads are issued before the block waits for the split scale
    const size_t i = size_t(bid_) * blockDim.x + threadIdx.x;
    const bool on = i < n;
    const float di = on ? d[i] : 0.0f;
    const float2 xv = on && !first ? x2[i] : make_float2(0.0f, 0.0f);
    __shared__ float2 sc;
    if (threadIdx.x == 0) sc = split(scale[0]);
    __syncthreads();
    if (!on) return;
    x2[i] = ff_add_scaled(xv, sc, di, first != 0);
}
__global__ void ff_axpy_kernel(float2 *__restrict__ x2, const float *__restrict__ d, const double *__restrict__ scale,
                               size_t n, int first) {
    pdl_wait();
    ff_axpy_kernel_impl(blockIdx.x, gridDim.x, x2, d, scale, n, first);
}
struct ff_axpy_kernel_args {
    int nb_;
    float2 *x2;
    const float *d;
    const double *scale;
    size_t n;
    int first;
};
__global__ void ff_axpy_kernel_multi(const __grid_constant__ MultiP<ff_axpy_kernel_args> M) {
    pdl_wait();
    int b_;
    const ff_axpy_kernel_args &q_ = M.a[merge_find(M.start, M.n, b_)];
    ff_axpy_kernel_impl(b_, q_.nb_, q_.x2, q_.d, q_.scale, q_.n, q_.first);
}
void ff_axpy_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, float2 *x2, const float *d,
                       const double *scale, size_t n, int first) {
    if (Recorder *r_ = batch_recorder()) {
        ff_axpy_kernel_args q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.x2 = x2;
        q_.d = d;
        q_.scale = scale;
        q_.n = n;
        q_.first = first;
        batch_record(r_, reinterpret_cast<const void *>(&ff_axpy_kernel_multi), q_, grid_, block_, smem_, kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &ff_axpy_kernel, grid_, block_, smem_, s_, x2, d, scale, n, first);
}

// The end of the last cycle of an inner solve of the mixed refinement, in one
// pass: y = R^-1 s for the leading k x k triangle of the rotated Hessenberg
// matrix (column-major, leading dimension ldh), solved by one thread of every
// block with the substitution of the separate triangular-solve kernel; d = x +
// sum_c y_c Z_c with the FP32 sums of the separate basis update (x null: the
// inner iterate is still zero); then the refinement iterate's pairs +=
// scale[0] * d as ff_axpy forms it (first: pairs = scale[0] * d).  The same
// values as those three kernels, bit for bit.  Each thread takes kFinU entries
// a block width apart.
constexpr int kFinU = 8;
__device__ __forceinline__ void ff_finish_kernel_impl(int bid_, int nb_, const double *__restrict__ Hm, int ldh,
                                                      const double *__restrict__ sv, int k,
                                                      const float *__restrict__ Z, size_t ld,
                                                      const float *__restrict__ x, float2 *__restrict__ x2,
                                                      const double *__restrict__ scale, size_t n, int first) {
    extern __shared__ double R[];          // k x k, R[i * k + l] = row i, column l
    __shared__ double sS[64], yS[64];
    __shared__ float cf[64];
    __shared__ float2 sc;
    __shared__ double scl;
    if (threadIdx.x == 0) scl = scale[0];
    // the entries' x first (they do not wait for y)
    const size_t base = size_t(bid_) * blockDim.x * kFinU + threadIdx.x;
    float acc[kFinU];
#pragma unroll
    for (int u = 0; u < kFinU; ++u) {
        const size_t i = base + size_t(u) * blockDim.x;
        acc[u] = (x && i < n) ? x[i] : 0.0f;
    }
    for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
        const int l = t / k, i = t % k;            // column l, row i
        if (i <= l) R[i * k + l] = Hm[size_t(l) * ldh + i];
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) sS[i] = sv[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = k - 1; i >= 0; --i) {
            double t = sS[i];
            for (int l = i + 1; l < k; ++l) t -= R[i * k + l] * yS[l];
            yS[i] = t / R[i * k + i];
        }
        sc = split(scl);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < k; i += blockDim.x) cf[i] = float(1.0 * yS[i]);
    __syncthreads();
    // basis vector by basis vector, kFinU independent loads each and two
    // vectors' loads in flight (each entry still adds its terms in the order
    // c = 0, 1, ...)
#pragma unroll 2
    for (int c = 0; c < k; ++c) {
        const float cc = cf[c];
        const float *Zc = Z + size_t(c) * ld;
#pragma unroll
        for (int u = 0; u < kFinU; ++u) {
            const size_t i = base + size_t(u) * blockDim.x;
            if (i < n) acc[u] = fma(cc, Zc[i], acc[u]);
        }
    }
#pragma unroll
    for (int u = 0; u < kFinU; ++u) {
        const size_t i = base + size_t(u) * blockDim.x;
        if (i < n) x2[i] = ff_add_scaled(first ? make_float2(0.0f, 0.0f) : x2[i], sc, acc[u], first != 0);
    }
}
__global__ void __launch_bounds__(256, 4) ff_finish_kernel(const double *__restrict__ Hm, int ldh,
                                                        const double *__restrict__ sv, int k,
                                                        const float *__restrict__ Z, size_t ld,
                                                        const float *__restrict__ x, float2 *__restrict__ x2,
                                                        const double *__restrict__ scale, size_t n, int first) {
    pdl_wait();
    ff_finish_kernel_impl(blockIdx.x, gridDim.x, Hm, ldh, sv, k, Z, ld, x, x2, scale, n, first);
}
struct ff_finish_kernel_args {
    int nb_;
    const double *Hm;
    int ldh;
    const double *sv;
    int k;
    const float *Z;
    size_t ld;
    const float *x;
    float2 *x2;
    const double *scale;
    size_t n;
    int first;
};
__global__ void __launch_bounds__(256, 4) ff_finish_kernel_multi(const __grid_constant__ MultiP<ff_finish_kernel_args> M) {
    pdl_wait();
    int b_;
    const ff_finish_kernel_args &q_ = M.a[merge_find(M.start, M.n, b_)];
    ff_finish_kernel_impl(b_, q_.nb_, q_.Hm, q_.ldh, q_.sv, q_.k, q_.Z, q_.ld, q_.x, q_.x2, q_.scale, q_.n, q_.first);
}
void ff_finish_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, const double *Hm, int ldh,
                         const double *sv, int k, const float *Z, size_t ld, const float *x, float2 *x2,
                         const double *scale, size_t n, int first) {
    if (Recorder *r_ = batch_recorder()) {
        ff_finish_kernel_args q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.Hm = Hm;
        q_.ldh = ldh;
        q_.sv = sv;
        q_.k = k;
        q_.Z = Z;
        q_.ld = ld;
        q_.x = x;
        q_.x2 = x2;
        q_.scale = scale;
        q_.n = n;
        q_.first = first;
        batch_record(r_, reinterpret_cast<const void *>(&ff_finish_kernel_multi), q_, grid_, block_, smem_,
                     kPdlKrylov);
        return;
    }
    pdl_launch(kPdlKrylov, &ff_finish_kernel, grid_, block_, smem_, s_, Hm, ldh, sv, k, Z, ld, x, x2, scale, n, first);
}

// a = b = hi + lo of the pairs, rounded once to FP64 (within 2^-53 of the
// pair's value); b may be null
__device__ __forceinline__ void ff_join_kernel_impl(int bid_, int nb_, const float2 *__restrict__ x2,
                                                    double *__restrict__ a, double *__restrict__ b, size_t n) {
    const size_t i = size_t(bid_) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 v = x2[i];
    const double r = double(v.x) + double(v.y);
    a[i] = r;
    if (b) b[i] = r;
}
__global__ void ff_join_kernel(const float2 *__restrict__ x2, double *__restrict__ a, double *__restrict__ b,
                               size_t n) {
    pdl_wait();
    ff_join_kernel_impl(blockIdx.x, gridDim.x, x2, a, b, n);
}
struct ff_join_kernel_args {
    int nb_;
    const float2 *x2;
    double *a;
    double *b;
    size_t n;
};
__global__ void ff_join_kernel_multi(const __grid_constant__ MultiP<ff_join_kernel_args> M) {
    pdl_wait();
    int b_;
    const ff_join_kernel_args &q_ = M.a[merge_find(M.start, M.n, b_)];
    ff_join_kernel_impl(b_, q_.nb_, q_.x2, q_.a, q_.b, q_.n);
}
void ff_join_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, const float2 *x2, double *a,
                       double *b, size_t n) {
    if (Recorder *r_ = batch_recorder()) {
        ff_join_kernel_args q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.x2 = x2;
        q_.a = a;
        q_.b = b;
        q_.n = n;
        batch_record(r_, reinterpret_cast<const void *>(&ff_join_kernel_multi), q_, grid_, block_, smem_, kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &ff_join_kernel, grid_, block_, smem_, s_, x2, a, b, n);
}


// r = b - S x with x given split; S split in the packed FP64 layout (element
// j of facet e in 16-byte group (j / 2, e), lane j % 2, here two float pairs)
// sum of a double over the block (fixed tree: warp shuffles, then warp 0 over
// the warp sums); every thread gets the block's sum in warp 0, the others
// their warp's
__device__ __forceinline__ double ff_block_sum(double v) {
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

// res = b - S x in two-float arithmetic (x as split pairs), one thread per
// facet row: a block takes kResFacets facets, thread (r, f) of it row r of
// facet f.  The threads first stage the pairs of their facets and of the four
// neighbours in shared memory (thread (r, f) component r of the five), then
// each adds the 5 (p+1) products of its row in the order of the packed layout.
// res may be null, and c32 names the FP32 start of an inner solve on res
// (F32Copy).  With partial non-null also ||res||^2: block sums of the rows'
// squares, the last block adding the block sums in block order into out[0]
// and handing the value to the host through pub (the value, a system fence,
// then seq).
constexpr int kResFacets = kResFFFacets;

template <int P>
__device__ __forceinline__ void residual_ff_kernel_impl(int bid_, int nb_, int NF, const float4 *__restrict__ S2,
                                                        const int32_t *__restrict__ nbr, const double *__restrict__ b,
                                                        const float2 *__restrict__ x2, double *__restrict__ res,
                                                        double *partial, unsigned int *counter, double *out,
                                                        HostValue *pub, int32_t seq, const F32Copy c32) {
    constexpr int PP = P + 1, RS = 5 * PP, NQR = (RS + 1) / 2;   // entries of a row, 16-byte groups it touches
    __shared__ float2 sx[5][PP][kResFacets];
    const int r = threadIdx.x / kResFacets, f = threadIdx.x % kResFacets, e = bid_ * kResFacets + f;
    const bool on = e < NF;
    if (on) {
        sx[0][r][f] = x2[size_t(r) * NF + e];
#pragma unroll
        for (int q = 1; q < 5; ++q) sx[q][r][f] = x2[size_t(r) * NF + __ldg(nbr + size_t(q - 1) * NF + e)];
    }
    __syncthreads();
    double sq = 0.0;
    if (on) {
        // row r holds entries j0 .. j0 + RS - 1, in groups q0 .. q0 + NQR - 1
        // (j0 is even whenever RS is, and the entry of lane g of group q0 + t
        // is then 2t + g of the row)
        const int j0 = r * RS, q0 = j0 / 2, odd = (RS % 2) ? (j0 & 1) : 0;
        float4 v[NQR];
#pragma unroll
        for (int t = 0; t < NQR; ++t) v[t] = __ldg(S2 + size_t(q0 + t) * NF + e);
        FFAcc acc;
#pragma unroll
        for (int t = 0; t < NQR; ++t) {
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                const int k = 2 * t + g - odd;
                if (k >= 0 && k < RS)
                    acc.add(g ? make_float2(v[t].z, v[t].w) : make_float2(v[t].x, v[t].y), sx[k / PP][k % PP][f]);
            }
        }
        const double rv = b[size_t(r) * NF + e] - acc.value();
        if (res) res[size_t(r) * NF + e] = rv;
        if (c32.b32) {
            c32.b32[size_t(r) * NF + e] = float(rv * c32.scale);
            c32.z32[size_t(r) * NF + e] = 0.0f;
        }
        sq = rv * rv;
    }
    if (!partial) return;
    __shared__ bool last;
    const double tot = ff_block_sum(sq);
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
    a = ff_block_sum(a);
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
__global__ void __launch_bounds__(kResFacets * (P + 1)) residual_ff_kernel(int NF, const float4 *__restrict__ S2,
                                                          const int32_t *__restrict__ nbr,
                                                          const double *__restrict__ b, const float2 *__restrict__ x2,
                                                          double *__restrict__ res, double *partial,
                                                          unsigned int *counter, double *out, HostValue *pub,
                                                          int32_t seq, const F32Copy c32) {
    pdl_wait();
    residual_ff_kernel_impl<P>(blockIdx.x, gridDim.x, NF, S2, nbr, b, x2, res, partial, counter, out, pub, seq, c32);
}
template <int P>
struct residual_ff_kernel_args {
    int nb_;
    int NF;
    const float4 *S2;
    const int32_t *nbr;
    const double *b;
    const float2 *x2;
    double *res;
    double *partial;
    unsigned int *counter;
    double *out;
    HostValue *pub;
    int32_t seq;
    F32Copy c32;
};
template <int P>
__global__ void __launch_bounds__(kResFacets * (P + 1)) residual_ff_kernel_multi(const __grid_constant__ MultiP<residual_ff_kernel_args<P>> M) {
    pdl_wait();
    int b_;
    const residual_ff_kernel_args<P> &q_ = M.a[merge_find(M.start, M.n, b_)];
    residual_ff_kernel_impl<P>(b_, q_.nb_, q_.NF, q_.S2, q_.nbr, q_.b, q_.x2, q_.res, q_.partial, q_.counter, q_.out,
                               q_.pub, q_.seq, q_.c32);
}
template <int P>
void residual_ff_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, int NF, const float4 *S2,
                           const int32_t *nbr, const double *b, const float2 *x2, double *res, double *partial,
                           unsigned int *counter, double *out, HostValue *pub, int32_t seq, const F32Copy &c32) {
    if (Recorder *r_ = batch_recorder()) {
        residual_ff_kernel_args<P> q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.NF = NF;
        q_.S2 = S2;
        q_.nbr = nbr;
        q_.b = b;
        q_.x2 = x2;
        q_.res = res;
        q_.partial = partial;
        q_.counter = counter;
        q_.out = out;
        q_.pub = pub;
        q_.seq = seq;
        q_.c32 = c32;
        batch_record(r_, reinterpret_cast<const void *>(&residual_ff_kernel_multi<P>), q_, grid_, block_, smem_,
                     kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &residual_ff_kernel<P>, grid_, block_, smem_, s_, NF, S2, nbr, b, x2, res, partial, counter,
               out, pub, seq, c32);
}


// (r_u, r_h may live in page-locked host memory read over the C2C link; with
// cu, ch non-null each value read is also stored there, in HBM)
template <int NP>
__device__ __forceinline__ void stage_cell_rhs(int N, int K0, const double *__restrict__ r_u,
                                               const double *__restrict__ r_h, float2 (*sIn)[kCellsPad],
                                               double *__restrict__ cu = nullptr, double *__restrict__ ch = nullptr) {
    const int nc = min(kCells, N - K0);
    for (int j = threadIdx.x; j < nc * 2 * NP; j += blockDim.x) {
        const size_t k = size_t(K0) * 2 * NP + j;
        const double v = r_u[k];
        if (cu) cu[k] = v;
        sIn[j % (2 * NP)][j / (2 * NP)] = split(v);
    }
    for (int j = threadIdx.x; j < nc * NP; j += blockDim.x) {
        const size_t k = size_t(K0) * NP + j;
        const double v = r_h[k];
        if (ch) ch[k] = v;
        sIn[2 * NP + j % NP][j / NP] = split(v);
    }
}

// the product of two pairs as a normalised pair (leading product by FMA with
// its exact error, the cross terms added to it; about 2^-46 relative)
__device__ __forceinline__ float2 ff_mul(const float2 a, const float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    const float hi = __fadd_rn(p, e);
    return make_float2(hi, __fsub_rn(e, __fsub_rn(hi, p)));
}

// Step 1 of a solve, keeping what step 3 needs: z_K = R_M r_K (= A_K^-1
// Mass_K r_K, the cell solution for lambda = 0) in two-float arithmetic, stored
// as normalised pairs (z2 [NK][N], when given), and the cell rows ycell =
// C_K z_K (= W_K r_K) formed from the cell's geometry instead of a stored
// W_K.  Row (i, j) of C_K (edge i, trace node j) is sum_b N_ibj (H t_y z_u[b]
// - H t_x z_v[b] + tau_s |e_i| z_h[b]) with t the edge vector and N_ibj =
// int_e phi_b mu_j, nonzero only for the cell nodes b on the edge: cgeo holds
// the pairs of H t_y, -H t_x, tau_s |e_i| per cell and edge ([N][3][3]), ctab_b
// / ctab_v the nodes and pairs of N per row ([3(p+1)][p+1]).  The block's 32
// cells are the lanes; the eight warps take the rows of R_M in turn, then the
// rows of C_K.
template <int P>
__device__ __forceinline__ void rhs_cell_z_kernel_impl(int bid_, int nb_, int N, const float4 *__restrict__ Rm2,
                                                       const float2 *__restrict__ cgeo,
                                                       const int32_t *__restrict__ ctab_b,
                                                       const float2 *__restrict__ ctab_v,
                                                       const double *__restrict__ r_u,
                                                       const double *__restrict__ r_h, double *__restrict__ ycell,
                                                       float2 *__restrict__ z2, double *__restrict__ cu,
                                                       double *__restrict__ ch) {
    constexpr int PP = P + 1, NP = (P + 1) * (P + 2) / 2, NK = 3 * NP, M = 3 * PP, NW = 8;
    constexpr int KP = (NK + 1) / 2, RW = (NK + NW - 1) / NW;
    __shared__ float2 sIn[NK][kCellsPad];      // r_K, then z_K
    __shared__ int32_t tb[M][PP];
    __shared__ float2 tv[M][PP];
    for (int t = threadIdx.x; t < M * PP; t += blockDim.x) {
        tb[t / PP][t % PP] = ctab_b[t];
        tv[t / PP][t % PP] = ctab_v[t];
    }
    const int K0 = bid_ * kCells, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    stage_cell_rhs<NP>(N, K0, r_u, r_h, sIn, cu, ch);
    __syncthreads();
    const int K = K0 + lane;
    const bool on = K < N;
    float2 zr[RW];
#pragma unroll
    for (int u = 0; u < RW; ++u) {
        const int rho = w + u * NW;
        zr[u] = make_float2(0.0f, 0.0f);
        if (on && rho < NK) {
            FFAcc acc;
            row_pairs<NK>(acc, Rm2 + (size_t(bid_) * NK * KP + size_t(rho) * KP) * kCells + lane, sIn, lane);
            const float hi = __fadd_rn(acc.s, acc.c);
            zr[u] = make_float2(hi, __fsub_rn(acc.c, __fsub_rn(hi, acc.s)));
        }
    }
    __syncthreads();                            // every warp has read r_K
#pragma unroll
    for (int u = 0; u < RW; ++u) {
        const int rho = w + u * NW;
        if (rho < NK) {
            sIn[rho][lane] = zr[u];
            if (z2 && on) z2[size_t(rho) * N + K] = zr[u];
        }
    }
    __syncthreads();
    if (!on) return;
    for (int t = w; t < M; t += NW) {
        const float2 *gc = cgeo + (size_t(K) * 3 + t / PP) * 3;
        const float2 g0 = gc[0], g1 = gc[1], g2 = gc[2];
        FFAcc acc;
#pragma unroll
        for (int q = 0; q < PP; ++q) {
            const int b = tb[t][q];
            const float2 v = tv[t][q];
            acc.add(ff_mul(v, g0), sIn[b][lane]);
            acc.add(ff_mul(v, g1), sIn[NP + b][lane]);
            acc.add(ff_mul(v, g2), sIn[2 * NP + b][lane]);
        }
        ycell[size_t(t) * N + K] = acc.value();
    }
}
template <int P>
__global__ void __launch_bounds__(256) rhs_cell_z_kernel(int N, const float4 *__restrict__ Rm2,
                                                         const float2 *__restrict__ cgeo,
                                                         const int32_t *__restrict__ ctab_b,
                                                         const float2 *__restrict__ ctab_v,
                                                         const double *__restrict__ r_u,
                                                         const double *__restrict__ r_h, double *__restrict__ ycell,
                                                         float2 *__restrict__ z2, double *__restrict__ cu,
                                                         double *__restrict__ ch) {
    pdl_wait();
    rhs_cell_z_kernel_impl<P>(blockIdx.x, gridDim.x, N, Rm2, cgeo, ctab_b, ctab_v, r_u, r_h, ycell, z2, cu, ch);
}
template <int P>
struct rhs_cell_z_kernel_args {
    int nb_;
    int N;
    const float4 *Rm2;
    const float2 *cgeo;
    const int32_t *ctab_b;
    const float2 *ctab_v;
    const double *r_u;
    const double *r_h;
    double *ycell;
    float2 *z2;
    double *cu;
    double *ch;
};
template <int P>
__global__ void __launch_bounds__(256) rhs_cell_z_kernel_multi(const __grid_constant__ MultiP<rhs_cell_z_kernel_args<P>> M) {
    pdl_wait();
    int b_;
    const rhs_cell_z_kernel_args<P> &q_ = M.a[merge_find(M.start, M.n, b_)];
    rhs_cell_z_kernel_impl<P>(b_, q_.nb_, q_.N, q_.Rm2, q_.cgeo, q_.ctab_b, q_.ctab_v, q_.r_u, q_.r_h, q_.ycell, q_.z2,
                              q_.cu, q_.ch);
}
template <int P>
void rhs_cell_z_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, int N, const float4 *Rm2,
                          const float2 *cgeo, const int32_t *ctab_b, const float2 *ctab_v, const double *r_u,
                          const double *r_h, double *ycell, float2 *z2, double *cu, double *ch) {
    if (Recorder *r_ = batch_recorder()) {
        rhs_cell_z_kernel_args<P> q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.N = N;
        q_.Rm2 = Rm2;
        q_.cgeo = cgeo;
        q_.ctab_b = ctab_b;
        q_.ctab_v = ctab_v;
        q_.r_u = r_u;
        q_.r_h = r_h;
        q_.ycell = ycell;
        q_.z2 = z2;
        q_.cu = cu;
        q_.ch = ch;
        batch_record(r_, reinterpret_cast<const void *>(&rhs_cell_z_kernel_multi<P>), q_, grid_, block_, smem_,
                     kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &rhs_cell_z_kernel<P>, grid_, block_, smem_, s_, N, Rm2, cgeo, ctab_b, ctab_v, r_u, r_h,
               ycell, z2, cu, ch);
}

// step 1, cell part: ycell[t][K] = sum_kappa W[t*NK + kappa][K] r_K[kappa]
template <int P>
__device__ __forceinline__ void rhs_cell_ff_kernel_impl(int bid_, int nb_, int N, const float4 *__restrict__ W2,
                                                        const double *__restrict__ r_u,
                                                        const double *__restrict__ r_h, double *__restrict__ ycell,
                                                        double *__restrict__ cu, double *__restrict__ ch) {
    constexpr int PP = P + 1, NP = (P + 1) * (P + 2) / 2, NK = 3 * NP, M = 3 * PP, NW = 4;
    constexpr int KP = (NK + 1) / 2;
    __shared__ float2 sIn[NK][kCellsPad];
    const int K0 = bid_ * kCells, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    stage_cell_rhs<NP>(N, K0, r_u, r_h, sIn, cu, ch);
    __syncthreads();
    const int K = K0 + lane;
    if (K >= N) return;
    for (int t = w; t < M; t += NW) {
        FFAcc acc;
        row_pairs<NK>(acc, W2 + (size_t(bid_) * M * KP + size_t(t) * KP) * kCells + lane, sIn, lane);
        ycell[size_t(t) * N + K] = acc.value();
    }
}
template <int P>
__global__ void __launch_bounds__(128, 8) rhs_cell_ff_kernel(int N, const float4 *__restrict__ W2,
                                                             const double *__restrict__ r_u,
                                                             const double *__restrict__ r_h,
                                                             double *__restrict__ ycell, double *__restrict__ cu,
                                                             double *__restrict__ ch) {
    pdl_wait();
    rhs_cell_ff_kernel_impl<P>(blockIdx.x, gridDim.x, N, W2, r_u, r_h, ycell, cu, ch);
}
template <int P>
struct rhs_cell_ff_kernel_args {
    int nb_;
    int N;
    const float4 *W2;
    const double *r_u;
    const double *r_h;
    double *ycell;
    double *cu;
    double *ch;
};
template <int P>
__global__ void __launch_bounds__(128, 8) rhs_cell_ff_kernel_multi(const __grid_constant__ MultiP<rhs_cell_ff_kernel_args<P>> M) {
    pdl_wait();
    int b_;
    const rhs_cell_ff_kernel_args<P> &q_ = M.a[merge_find(M.start, M.n, b_)];
    rhs_cell_ff_kernel_impl<P>(b_, q_.nb_, q_.N, q_.W2, q_.r_u, q_.r_h, q_.ycell, q_.cu, q_.ch);
}
template <int P>
void rhs_cell_ff_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, int N, const float4 *W2,
                           const double *r_u, const double *r_h, double *ycell, double *cu, double *ch) {
    if (Recorder *r_ = batch_recorder()) {
        rhs_cell_ff_kernel_args<P> q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.N = N;
        q_.W2 = W2;
        q_.r_u = r_u;
        q_.r_h = r_h;
        q_.ycell = ycell;
        q_.cu = cu;
        q_.ch = ch;
        batch_record(r_, reinterpret_cast<const void *>(&rhs_cell_ff_kernel_multi<P>), q_, grid_, block_, smem_, kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &rhs_cell_ff_kernel<P>, grid_, block_, smem_, s_, N, W2, r_u, r_h, ycell, cu, ch);
}


// step 3: q_K = R_M r_K - X_B lambda_K, written in the caller's u / h layout
template <int P>
__global__ void __launch_bounds__(256) recover_ff_kernel(int N, int NF, const float4 *__restrict__ Rm2,
                                                         const float4 *__restrict__ Xb2, const double *__restrict__ r_u,
                                                         const double *__restrict__ r_h, const double *__restrict__ lam,
                                                         const int32_t *__restrict__ facet_of,
                                                         const int32_t *__restrict__ flip, double *__restrict__ u,
                                                         double *__restrict__ hout) {
    constexpr int PP = P + 1, NP = (P + 1) * (P + 2) / 2, NK = 3 * NP, M = 3 * PP, NW = 8;
    constexpr int KP = (NK + 1) / 2, MP = (M + 1) / 2;
    __shared__ float2 sIn[NK + M][kCellsPad];   // r_K, then lambda on the cell's three facets
    __shared__ double sOut[NK][kCellsPad];
    const int K0 = blockIdx.x * kCells, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nc = min(kCells, N - K0);
    stage_cell_rhs<NP>(N, K0, r_u, r_h, sIn);
    for (int j = threadIdx.x; j < nc * M; j += blockDim.x) {
        const int cell = j / M, q = j % M, i = q / PP, jj = q % PP, K = K0 + cell;
        const int f = facet_of[3 * K + i], fl = flip[3 * K + i];
        sIn[NK + q][cell] = split(lam[size_t(fl ? P - jj : jj) * NF + f]);
    }
    __syncthreads();
    const int K = K0 + lane;
    if (K < N) {
        for (int rho = w; rho < NK; rho += NW) {
            FFAcc acc;
            row_pairs<NK>(acc, Rm2 + (size_t(blockIdx.x) * NK * KP + size_t(rho) * KP) * kCells + lane, sIn, lane);
            row_pairs<M>(acc, Xb2 + (size_t(blockIdx.x) * NK * MP + size_t(rho) * MP) * kCells + lane, sIn + NK,
                         lane, true);
            sOut[rho][lane] = acc.value();
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < nc * 2 * NP; j += blockDim.x)
        u[size_t(K0) * 2 * NP + j] = sOut[j % (2 * NP)][j / (2 * NP)];
    for (int j = threadIdx.x; j < nc * NP; j += blockDim.x) hout[size_t(K0) * NP + j] = sOut[2 * NP + j % NP][j / NP];
}

// step 3 from the kept z_K: q_K = z_K - X_B lambda_K (two-float, z as the
// starting sum), written in the caller's u / h layout
template <int P>
__global__ void __launch_bounds__(256) recover_z_kernel(int N, int NF, const float2 *__restrict__ z2,
                                                        const float4 *__restrict__ Xb2,
                                                        const double *__restrict__ lam,
                                                        const int32_t *__restrict__ facet_of,
                                                        const int32_t *__restrict__ flip, double *__restrict__ u,
                                                        double *__restrict__ hout) {
    constexpr int PP = P + 1, NP = (P + 1) * (P + 2) / 2, NK = 3 * NP, M = 3 * PP, NW = 8;
    constexpr int MP = (M + 1) / 2;
    __shared__ float2 sIn[M][kCellsPad];        // lambda on the cell's three facets
    __shared__ double sOut[NK][kCellsPad];
    const int K0 = blockIdx.x * kCells, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nc = min(kCells, N - K0);
    for (int j = threadIdx.x; j < nc * M; j += blockDim.x) {
        const int cell = j / M, q = j % M, i = q / PP, jj = q % PP, K = K0 + cell;
        const int f = facet_of[3 * K + i], fl = flip[3 * K + i];
        sIn[q][cell] = split(lam[size_t(fl ? P - jj : jj) * NF + f]);
    }
    __syncthreads();
    const int K = K0 + lane;
    if (K < N) {
        for (int rho = w; rho < NK; rho += NW) {
            FFAcc acc;
            const float2 z = z2[size_t(rho) * N + K];
            acc.s = z.x;
            acc.c = z.y;
            row_pairs<M>(acc, Xb2 + (size_t(blockIdx.x) * NK * MP + size_t(rho) * MP) * kCells + lane, sIn, lane,
                         true);
            sOut[rho][lane] = acc.value();
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < nc * 2 * NP; j += blockDim.x)
        u[size_t(K0) * 2 * NP + j] = sOut[j % (2 * NP)][j / (2 * NP)];
    for (int j = threadIdx.x; j < nc * NP; j += blockDim.x) hout[size_t(K0) * NP + j] = sOut[2 * NP + j % NP][j / NP];
}

}  // namespace

cudaError_t launch_split(const double *a, float2 *out, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    split_kernel<<<blocks(n, 256), 256, 0, s>>>(a, out, n);
    return cudaGetLastError();
}

cudaError_t launch_split_pairs(const double *a, float2 *out, int rows, int cols, size_t N, cudaStream_t s) {
    const size_t n = size_t(rows) * ((cols + 1) / 2) * N;
    if (n == 0) return cudaSuccess;
    split_pairs_kernel<<<blocks(n, 256), 256, 0, s>>>(a, reinterpret_cast<float4 *>(out), rows, cols, N);
    return cudaGetLastError();
}

cudaError_t launch_ff_axpy(float2 *x2, const float *d, const double *scale, size_t n, bool first, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    ff_axpy_kernel_go(blocks(n, 256), 256, 0, s, x2, d, scale, n, first ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_ff_finish(const double *Hm, int ldh, const double *sv, int k, const float *Z, size_t ld,
                             const float *x, float2 *x2, const double *scale, size_t n, bool first, cudaStream_t s) {
    if (n == 0 || k <= 0) return cudaSuccess;
    if (k > 64) return cudaErrorInvalidValue;
    const size_t per = size_t(256) * kFinU;
    ff_finish_kernel_go(unsigned((n + per - 1) / per), 256, sizeof(double) * size_t(k) * k, s, Hm, ldh, sv, k, Z, ld,
                        x, x2, scale, n, first ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_ff_join(const float2 *x2, double *a, double *b, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    ff_join_kernel_go(blocks(n, 256), 256, 0, s, x2, a, b, n);
    return cudaGetLastError();
}

cudaError_t launch_residual_ff(hdg_handle *h, const double *b, const float2 *x2, double *res, double *partial,
                               unsigned int *counter, double *out, HostValue *pub, int32_t seq, const F32Copy &c32) {
    HDG_DISPATCH_P(h->p, (residual_ff_kernel_go<P>(blocks(h->NF, kResFacets), kResFacets * (P + 1), 0, h->stream, h->NF,
                                                   reinterpret_cast<const float4 *>(h->d_Sval2), h->d_nbr, b, x2, res,
                                                   partial, counter, out, pub, seq, c32)));
    return cudaGetLastError();
}

cudaError_t launch_rhs_ff(hdg_handle *h, const double *r_u, const double *r_h, double *g, double *ycell,
                          double *copy_u, double *copy_h, const NormOut &nrm) {
    HDG_DISPATCH_P(h->p, (rhs_cell_ff_kernel_go<P>(blocks(h->N, kCells), 128, 0, h->stream, h->N, reinterpret_cast<const float4 *>(h->d_W2), r_u, r_h,
                                                                                               ycell, copy_u, copy_h)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_rhs_gather(h, ycell, g, nrm);
}

cudaError_t launch_rhs_z(hdg_handle *h, const double *r_u, const double *r_h, double *g, double *ycell, float2 *z2,
                         double *copy_u, double *copy_h, const NormOut &nrm) {
    HDG_DISPATCH_P(h->p, (rhs_cell_z_kernel_go<P>(blocks(h->N, kCells), 256, 0, h->stream, h->N,
                                                  reinterpret_cast<const float4 *>(h->d_Rm2), h->d_cgeo, h->d_ctab_b,
                                                  h->d_ctab_v, r_u, r_h, ycell, z2, copy_u, copy_h)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_rhs_gather(h, ycell, g, nrm);
}

cudaError_t launch_recover_z(hdg_handle *h, const float2 *z2, const double *lam, double *u, double *hout) {
    HDG_DISPATCH_P(h->p, (recover_z_kernel<P><<<blocks(h->N, kCells), 256, 0, h->stream>>>(
                             h->N, h->NF, z2, reinterpret_cast<const float4 *>(h->d_Xb2), lam, h->d_facet_of,
                             h->d_flip, u, hout)));
    return cudaGetLastError();
}

cudaError_t launch_recover_ff(hdg_handle *h, const double *r_u, const double *r_h, const double *lam, double *u,
                              double *hout) {
    HDG_DISPATCH_P(h->p, (recover_ff_kernel<P><<<blocks(h->N, kCells), 256, 0, h->stream>>>(
                             h->N, h->NF, reinterpret_cast<const float4 *>(h->d_Rm2),
                             reinterpret_cast<const float4 *>(h->d_Xb2), r_u, r_h, lam, h->d_facet_of, h->d_flip, u,
                             hout)));
    return cudaGetLastError();
}

}  // namespace hdg
