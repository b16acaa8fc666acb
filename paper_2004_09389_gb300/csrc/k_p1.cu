// Geometric V-cycle on the nested P1 levels for the coarse problem of the
// two-level method (Eq. coarse_problem_upwind): damped Jacobi smoothing with
// the level operators in padded row-major ELL form (width W a multiple of 4,
// slot q of row i at i * W + q), restriction by the transpose of the midpoint
// prolongation, and a dense inverse on the coarsest level.  A row's columns
// and values load as 16-byte vectors; its W products are summed in slot order.
#include "common.h"

namespace hdg {

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
__global__ void jacobi_kernel(int n, int W, const int32_t *__restrict__ col, const T *__restrict__ A,
                              const T *__restrict__ dinv, const T *__restrict__ b, const T *__restrict__ x,
                              T *__restrict__ xout, T omega, int first) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (first) {
        xout[i] = omega * dinv[i] * b[i];
        return;
    }
    const T ax = ell_row(i, W, col, A, x);
    xout[i] = fma(omega * dinv[i], b[i] - ax, x[i]);
}

template <typename T>
__global__ void residual_kernel(int n, int W, const int32_t *__restrict__ col, const T *__restrict__ A,
                                const T *__restrict__ b, const T *__restrict__ x, T *__restrict__ r) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    r[i] = b[i] - ell_row(i, W, col, A, x);
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


// Going down one level, fused: b_c = R (b_f - A_f x_f) with the fine residual
// formed on the fly for each child, and the first pre-smoothing sweep of the
// coarse level from zero, x_c = omega D_c^-1 b_c (skipped when xc is null).
// Eight lanes per coarse vertex share its children; their partial sums are
// combined by a fixed shuffle tree (deterministic).
template <typename T>
__global__ void __launch_bounds__(256) down_kernel(int nc, const int32_t *__restrict__ cp,
                                                   const int32_t *__restrict__ ci, const T *__restrict__ cw,
                                                   int nf, int W, const int32_t *__restrict__ col,
                                                   const T *__restrict__ A, const T *__restrict__ bf,
                                                   const T *__restrict__ xf, const T *__restrict__ dinv_c, T omega,
                                                   T *__restrict__ bc, T *__restrict__ xc) {
    const int gid = (blockIdx.x * blockDim.x + threadIdx.x) >> 3, lane = threadIdx.x & 7;
    const bool valid = gid < nc;
    T acc = T(0);
    if (valid) {
        for (int k = cp[gid] + lane; k < cp[gid + 1]; k += 8) {
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

// Going up one level, fused: x' = x + P e_c (midpoint prolongation, formed on
// the fly for every column) followed by one damped Jacobi sweep on x'.
template <typename T>
__global__ void up_kernel(int nf, int W, const int32_t *__restrict__ col, const T *__restrict__ A,
                          const T *__restrict__ dinv, const T *__restrict__ b, const T *__restrict__ x,
                          const int32_t *__restrict__ parent, const T *__restrict__ ec, T *__restrict__ xout,
                          T omega) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    T ax = T(0);
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
    const int a = parent[2 * i], bb = parent[2 * i + 1];
    const T xi = x[i] + ((a == bb) ? ec[a] : T(0.5) * (ec[a] + ec[bb]));
    xout[i] = fma(omega * dinv[i], b[i] - ax, xi);
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

__host__ __device__ constexpr size_t pad16(size_t bytes) { return (bytes + 15) / 16 * 16; }

// Shared-memory addresses and sizes of one tail level.  The table lives in
// shared memory (filled from the staged header, one thread per level) so that
// run-time level indices never put per-thread pointer arrays on the stack.
template <typename T>
struct TailSlot {
    T *A, *D, *cw, *x, *x2, *b, *r;
    int32_t *col, *cp, *ci, *par;
    int nv, nnz, nci, W;
};

// x_j + (P e_c)_j: the midpoint prolongation of the coarse correction added on the fly
template <typename T>
__device__ __forceinline__ T prolonged(const int32_t *par, const T *x, const T *ec, int j) {
    const int p0 = par[2 * j], p1 = par[2 * j + 1];
    return x[j] + ((p0 == p1) ? ec[p0] : T(0.5) * (ec[p0] + ec[p1]));
}

template <typename T>
__global__ void __launch_bounds__(1024, 1) tail_kernel(TailArgs a) {
    extern __shared__ __align__(16) unsigned char tail_smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ TailSlot<T> L[kTailMaxLevels];
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
    const T om = T(a.omega);
    // meanwhile, with plain loads into the scratch space after the image: the
    // first level's right-hand side and its first pre-smoothing sweep from
    // zero, x = omega D^-1 b (the inverse diagonal read from global memory)
    {
        const T *btop = static_cast<const T *>(a.b_top);
        const T *d0 = static_cast<const T *>(a.dinv0);
        T *b0 = reinterpret_cast<T *>(tail_smem + a.ob0), *x0 = reinterpret_cast<T *>(tail_smem + a.ox0);
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
    if (tid < a.nlev) {
        const TailHdr H = reinterpret_cast<const TailHdr *>(tail_smem)[tid];
        TailSlot<T> &S = L[tid];
        S.nv = H.nv; S.nnz = H.nnz; S.nci = H.nci; S.W = H.W;
        S.A = reinterpret_cast<T *>(tail_smem + H.oA);
        S.D = reinterpret_cast<T *>(tail_smem + H.oD);
        S.cw = reinterpret_cast<T *>(tail_smem + H.ocw);
        S.col = reinterpret_cast<int32_t *>(tail_smem + H.ocol);
        S.cp = reinterpret_cast<int32_t *>(tail_smem + H.ocp);
        S.ci = reinterpret_cast<int32_t *>(tail_smem + H.oci);
        S.par = reinterpret_cast<int32_t *>(tail_smem + H.opar);
        S.x = reinterpret_cast<T *>(tail_smem + H.ox);
        S.x2 = reinterpret_cast<T *>(tail_smem + H.ox2);
        S.b = reinterpret_cast<T *>(tail_smem + H.ob);
        S.r = reinterpret_cast<T *>(tail_smem + H.orr);
    }
    __syncthreads();
    const int nc = L[a.nlev - 1].nv;
    const double *sinv = a.inv_off >= 0 ? reinterpret_cast<const double *>(tail_smem + a.inv_off) : nullptr;
    const int last = a.nlev - 1;
    // ---- down: x holds the first sweep (or zero) on entry to each level
    for (int l = 0; l < last; ++l) {
        const int nv = L[l].nv, W = L[l].W;
        const int32_t *cl = L[l].col;
        const T *A = L[l].A, *D = L[l].D, *b = L[l].b;
        T *x = L[l].x, *x2 = L[l].x2, *r = L[l].r;
        for (int k = 1; k < a.nu1; ++k) {
            for (int i = tid; i < nv; i += nt) x2[i] = fma(om * D[i], b[i] - ell_row(i, W, cl, A, x), x[i]);
            __syncthreads();
            T *t = x; x = x2; x2 = t;
        }
        for (int i = tid; i < nv; i += nt) r[i] = b[i] - ell_row(i, W, cl, A, x);
        if (tid == 0) { L[l].x = x; L[l].x2 = x2; }   // read again only after later barriers
        __syncthreads();
        // restriction, with the coarse level's first sweep from zero
        const int ncv = L[l + 1].nv;
        const int32_t *cp = L[l + 1].cp, *ci = L[l + 1].ci;
        const T *cw = L[l + 1].cw, *Dc = L[l + 1].D;
        T *bc = L[l + 1].b, *xc = L[l + 1].x;
        const bool smooth_c = l + 1 < last;
        for (int i = tid; i < ncv; i += nt) {
            T acc = T(0);
            for (int k = cp[i]; k < cp[i + 1]; ++k) acc = fma(cw[k], r[ci[k]], acc);
            bc[i] = acc;
            if (smooth_c) xc[i] = a.nu1 == 0 ? T(0) : om * Dc[i] * acc;
        }
        __syncthreads();
    }
    // ---- coarsest: dense FP64 inverse, FP64 sums in every precision; four
    // lanes per row (FP64 arithmetic is a narrow pipe: few adds in the tree),
    // each summing every fourth column, combined by a fixed two-step shuffle
    {
        const double *inv = sinv ? sinv : a.inv;
        const T *b = L[last].b;
        T *x = L[last].x;
        const int sub = tid & 3, ng = nt >> 2;
        // whole warps take part in every shuffle: the row loop runs to a multiple of 8
        for (int i = tid >> 2; i < ((nc + 7) & ~7); i += ng) {
            double acc = 0.0;
            if (i < nc)
                for (int j = sub; j < nc; j += 4) acc = fma(inv[size_t(i) * nc + j], double(b[j]), acc);
            acc += __shfl_xor_sync(0xffffffffu, acc, 2);
            acc += __shfl_xor_sync(0xffffffffu, acc, 1);
            if (i < nc && sub == 0) x[i] = T(acc);
        }
        __syncthreads();
    }
    // ---- up: x += P e_c in place (a separate step: forming it on the fly in
    // the sweep multiplies the shared-memory gathers), then post-smoothing
    const T *ec = L[last].x;
    for (int l = last - 1; l >= 0; --l) {
        const int nv = L[l].nv, W = L[l].W;
        const int32_t *cl = L[l].col, *par = L[l + 1].par;
        const T *A = L[l].A, *D = L[l].D, *b = L[l].b;
        T *x = L[l].x, *x2 = L[l].x2;
        for (int i = tid; i < nv; i += nt) x[i] = prolonged(par, x, ec, i);
        __syncthreads();
        for (int k = 0; k < a.nu2; ++k) {
            for (int i = tid; i < nv; i += nt) x2[i] = fma(om * D[i], b[i] - ell_row(i, W, cl, A, x), x[i]);
            __syncthreads();
            T *t = x; x = x2; x2 = t;
        }
        ec = x;
    }
    T *xtop = static_cast<T *>(a.x_top);
    for (int i = tid; i < L[0].nv; i += nt) xtop[i] = ec[i];
}

}  // namespace

template <typename T>
cudaError_t launch_p1_jacobi(const DevLevel &L, const T *A, const T *dinv, const T *b, const T *x, T *xout, T omega,
                             bool first, cudaStream_t s) {
    jacobi_kernel<T><<<blocks(L.nv, 256), 256, 0, s>>>(L.nv, L.width, L.col, A, dinv, b, x, xout, omega, first ? 1 : 0);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_p1_residual(const DevLevel &L, const T *A, const T *b, const T *x, T *r, cudaStream_t s) {
    residual_kernel<T><<<blocks(L.nv, 256), 256, 0, s>>>(L.nv, L.width, L.col, A, b, x, r);
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

template <typename T>
cudaError_t launch_p1_down(const DevLevel &fine, const DevLevel &coarse, const T *A_f, const T *b_f, const T *x_f,
                           const T *dinv_c, T omega, T *b_c, T *x_c, cudaStream_t s) {
    const T *cw = sizeof(T) == 4 ? reinterpret_cast<const T *>(coarse.child_w32) : reinterpret_cast<const T *>(coarse.child_w);
    down_kernel<T><<<blocks(size_t(coarse.nv) * 8, 256), 256, 0, s>>>(coarse.nv, coarse.child_ptr, coarse.child_idx, cw,
                                                                      fine.nv, fine.width, fine.col, A_f, b_f, x_f, dinv_c,
                                                                      omega, b_c, x_c);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_p1_up(const DevLevel &fine, const DevLevel &coarse, const T *A_f, const T *dinv_f, const T *b_f,
                         const T *x_f, const T *ec, T *xout, T omega, cudaStream_t s) {
    up_kernel<T><<<blocks(fine.nv, 256), 256, 0, s>>>(fine.nv, fine.width, fine.col, A_f, dinv_f, b_f, x_f,
                                                      coarse.parent, ec, xout, omega);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_p1_tail(const TailArgs &a, size_t smem, cudaStream_t s) {
    // one fixed limit for every handle: the attribute is process-wide, so a
    // per-handle value could be lowered by another thread between set and launch
    if (smem > kTailSmemMax) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(tail_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kTailSmemMax));
    if (e != cudaSuccess) return e;
    tail_kernel<T><<<1, 1024, smem, s>>>(a);
    return cudaGetLastError();
}

#define HDG_P1_INST(T)                                                                                         \
    template cudaError_t launch_p1_jacobi<T>(const DevLevel &, const T *, const T *, const T *, const T *, T *, \
                                             T, bool, cudaStream_t);                                           \
    template cudaError_t launch_p1_residual<T>(const DevLevel &, const T *, const T *, const T *, T *,           \
                                               cudaStream_t);                                                  \
    template cudaError_t launch_p1_restrict<T>(const DevLevel &, const T *, T *, cudaStream_t);                 \
    template cudaError_t launch_p1_prolong_add<T>(const DevLevel &, int, const T *, T *, cudaStream_t);         \
    template cudaError_t launch_dense_apply<T>(const T *, int, const T *, T *, cudaStream_t);                  \
    template cudaError_t launch_p1_down<T>(const DevLevel &, const DevLevel &, const T *, const T *, const T *,  \
                                           const T *, T, T *, T *, cudaStream_t);                               \
    template cudaError_t launch_p1_up<T>(const DevLevel &, const DevLevel &, const T *, const T *, const T *,    \
                                         const T *, const T *, T *, T, cudaStream_t);                           \
    template cudaError_t launch_p1_tail<T>(const TailArgs &, size_t, cudaStream_t);
HDG_P1_INST(double)
HDG_P1_INST(float)

}  // namespace hdg
