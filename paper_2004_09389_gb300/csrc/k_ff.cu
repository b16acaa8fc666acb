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

// launch family of this file for pdl_launch (facet-row kernels)
constexpr unsigned kPdlFamily = 1;

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

// x += scale * d (refinement correction, FP32 -> FP64) and its split copy
__device__ __forceinline__ void axpby_split_kernel_impl(int bid_, int nb_, double *__restrict__ x,
                                                        float2 *__restrict__ x2, const float *__restrict__ d,
                                                        const double *__restrict__ scale, size_t n) {
    const size_t i = size_t(bid_) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = fma(scale[0], double(d[i]), x[i]);
    x[i] = v;
    x2[i] = split(v);
}
__global__ void axpby_split_kernel(double *__restrict__ x, float2 *__restrict__ x2, const float *__restrict__ d,
                                   const double *__restrict__ scale, size_t n) {
    pdl_wait();
    axpby_split_kernel_impl(blockIdx.x, gridDim.x, x, x2, d, scale, n);
}
struct axpby_split_kernel_args {
    int nb_;
    double *x;
    float2 *x2;
    const float *d;
    const double *scale;
    size_t n;
};
__global__ void axpby_split_kernel_multi(const __grid_constant__ MultiP<axpby_split_kernel_args> M) {
    pdl_wait();
    int b_;
    const axpby_split_kernel_args &q_ = M.a[merge_find(M.start, M.n, b_)];
    axpby_split_kernel_impl(b_, q_.nb_, q_.x, q_.x2, q_.d, q_.scale, q_.n);
}
void axpby_split_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, double *x, float2 *x2,
                           const float *d, const double *scale, size_t n) {
    if (Recorder *r_ = batch_recorder()) {
        axpby_split_kernel_args q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.x = x;
        q_.x2 = x2;
        q_.d = d;
        q_.scale = scale;
        q_.n = n;
        batch_record(r_, reinterpret_cast<const void *>(&axpby_split_kernel_multi), q_, grid_, block_, smem_, kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &axpby_split_kernel, grid_, block_, smem_, s_, x, x2, d, scale, n);
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

// res = b - S x in two-float arithmetic (x as split pairs); with partial
// non-null also ||res||^2: per-thread double sums, block sums, the last block
// adding the block sums in block order into out[0] and handing the value to
// the host through pub (the value, a system fence, then seq)
template <int P>
__device__ __forceinline__ void residual_ff_kernel_impl(int bid_, int nb_, int NF, const float4 *__restrict__ S2,
                                                        const int32_t *__restrict__ nbr, const double *__restrict__ b,
                                                        const float2 *__restrict__ x2, double *__restrict__ res,
                                                        double *partial, unsigned int *counter, double *out,
                                                        HostValue *pub, int32_t seq) {
    constexpr int PP = P + 1, NS = 5 * PP * PP, NQ = (NS + 1) / 2;
    const int e = bid_ * blockDim.x + threadIdx.x;
    double sq = 0.0;
    if (e < NF) {
        int src[5];
        src[0] = e;
#pragma unroll
        for (int q = 1; q < 5; ++q) src[q] = __ldg(nbr + size_t(q - 1) * NF + e);
        float2 xs[5][PP];
#pragma unroll
        for (int q = 0; q < 5; ++q)
#pragma unroll
            for (int c = 0; c < PP; ++c) xs[q][c] = x2[size_t(c) * NF + src[q]];
        FFAcc acc[PP];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const float4 v = __ldg(S2 + size_t(q) * NF + e);
            const float2 a[2] = {make_float2(v.x, v.y), make_float2(v.z, v.w)};
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                const int j = 2 * q + g;
                if (j < NS) {
                    const int r = j / (5 * PP), rem = j % (5 * PP);
                    acc[r].add(a[g], xs[rem / PP][rem % PP]);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < PP; ++r) {
            const double rv = b[size_t(r) * NF + e] - acc[r].value();
            res[size_t(r) * NF + e] = rv;
            sq = fma(rv, rv, sq);
        }
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
        if (pub) {
            pub->v = a;
            __threadfence_system();
            *reinterpret_cast<volatile int32_t *>(&pub->seq) = seq;
        }
    }
}
template <int P>
__global__ void __launch_bounds__(256) residual_ff_kernel(int NF, const float4 *__restrict__ S2,
                                                          const int32_t *__restrict__ nbr,
                                                          const double *__restrict__ b, const float2 *__restrict__ x2,
                                                          double *__restrict__ res, double *partial,
                                                          unsigned int *counter, double *out, HostValue *pub,
                                                          int32_t seq) {
    pdl_wait();
    residual_ff_kernel_impl<P>(blockIdx.x, gridDim.x, NF, S2, nbr, b, x2, res, partial, counter, out, pub, seq);
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
};
template <int P>
__global__ void __launch_bounds__(256) residual_ff_kernel_multi(const __grid_constant__ MultiP<residual_ff_kernel_args<P>> M) {
    pdl_wait();
    int b_;
    const residual_ff_kernel_args<P> &q_ = M.a[merge_find(M.start, M.n, b_)];
    residual_ff_kernel_impl<P>(b_, q_.nb_, q_.NF, q_.S2, q_.nbr, q_.b, q_.x2, q_.res, q_.partial, q_.counter, q_.out,
                               q_.pub, q_.seq);
}
template <int P>
void residual_ff_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, int NF, const float4 *S2,
                           const int32_t *nbr, const double *b, const float2 *x2, double *res, double *partial,
                           unsigned int *counter, double *out, HostValue *pub, int32_t seq) {
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
        batch_record(r_, reinterpret_cast<const void *>(&residual_ff_kernel_multi<P>), q_, grid_, block_, smem_,
                     kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &residual_ff_kernel<P>, grid_, block_, smem_, s_, NF, S2, nbr, b, x2, res, partial, counter,
               out, pub, seq);
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

cudaError_t launch_axpby_split(double *x, float2 *x2, const float *d, const double *scale, size_t n, cudaStream_t s) {
    axpby_split_kernel_go(blocks(n, 256), 256, 0, s, x, x2, d, scale, n);
    return cudaGetLastError();
}

cudaError_t launch_residual_ff(hdg_handle *h, const double *b, const float2 *x2, double *res, double *partial,
                               unsigned int *counter, double *out, HostValue *pub, int32_t seq) {
    HDG_DISPATCH_P(h->p, (residual_ff_kernel_go<P>(blocks(h->NF, 256), 256, 0, h->stream, h->NF,
                                                   reinterpret_cast<const float4 *>(h->d_Sval2), h->d_nbr, b, x2, res,
                                                   partial, counter, out, pub, seq)));
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

cudaError_t launch_recover_ff(hdg_handle *h, const double *r_u, const double *r_h, const double *lam, double *u,
                              double *hout) {
    HDG_DISPATCH_P(h->p, (recover_ff_kernel<P><<<blocks(h->N, kCells), 256, 0, h->stream>>>(
                             h->N, h->NF, reinterpret_cast<const float4 *>(h->d_Rm2),
                             reinterpret_cast<const float4 *>(h->d_Xb2), r_u, r_h, lam, h->d_facet_of, h->d_flip, u,
                             hout)));
    return cudaGetLastError();
}

}  // namespace hdg
