// Learned facet-patch smoother (an extension beyond the paper, which has none).
//
// For a trace residual r, facet e gets the features
//   X_e = (r_e, r_n1, ..., r_n4) / s_e,   s_e = RMS of those 5(p+1) values
// (its own p+1 values, then the four facets sharing a cell with it, in the
// order of the facet-row operator's neighbour list), a two-hidden-layer tanh
// network
//   y_e = W3 tanh(W2 tanh(W1 X_e + b1) + b2) + b3 + omega X_e[0:p+1]
// and the correction c_e = D_e^-1 (s_e y_e).  With zero weights this is the
// damped block-Jacobi step; the correction is positively homogeneous in r.
// Training minimises L = mean_b ||r_b - S c(r_b)||^2 / ||r_b||^2; the gradient
// with respect to c is -2 S^T (r - S c) / ||r||^2.
// Parameters theta = [W1 (HID x F) | b1 | W2 (HID x HID) | b2 | W3 (PP x HID) | b3],
// row-major, FP32; trace vectors in the internal layout x[r * NF + e].
#include "common.h"

namespace hdg {

namespace {

inline unsigned blocks(size_t n, int bs) { return unsigned((n + bs - 1) / bs); }

template <int P, int HID>
struct LN {
    static constexpr int PP = P + 1, F = 5 * PP;
    static constexpr int oW1 = 0, ob1 = oW1 + HID * F, oW2 = ob1 + HID, ob2 = oW2 + HID * HID, oW3 = ob2 + HID,
                         ob3 = oW3 + PP * HID, NPAR = ob3 + PP;
};

// features of facet e: X (normalised) and the scale s
template <int P>
__device__ __forceinline__ float patch_features(const int32_t *__restrict__ nbr, const float *__restrict__ r, int e,
                                                size_t NF, float (&X)[5 * (P + 1)]) {
    constexpr int PP = P + 1;
    int src[5];
    src[0] = e;
#pragma unroll
    for (int b = 1; b < 5; ++b) src[b] = __ldg(nbr + size_t(b - 1) * NF + e);
    float ss = 0.f;
#pragma unroll
    for (int b = 0; b < 5; ++b)
#pragma unroll
        for (int c = 0; c < PP; ++c) {
            const float v = r[size_t(c) * NF + src[b]];
            X[b * PP + c] = v;
            ss = fmaf(v, v, ss);
        }
    const float s = sqrtf(ss / float(5 * PP)) + 1e-30f;
    const float inv = 1.f / s;
#pragma unroll
    for (int i = 0; i < 5 * PP; ++i) X[i] *= inv;
    return s;
}

template <int P, int HID>
__device__ __forceinline__ void mlp(const float *__restrict__ th, const float (&X)[5 * (P + 1)], float omega,
                                    float (&h1)[HID], float (&h2)[HID], float (&y)[P + 1]) {
    using L = LN<P, HID>;
#pragma unroll 4
    for (int j = 0; j < HID; ++j) {
        float a = th[L::ob1 + j];
#pragma unroll
        for (int i = 0; i < L::F; ++i) a = fmaf(th[L::oW1 + j * L::F + i], X[i], a);
        h1[j] = tanhf(a);
    }
#pragma unroll 4
    for (int j = 0; j < HID; ++j) {
        float a = th[L::ob2 + j];
#pragma unroll
        for (int i = 0; i < HID; ++i) a = fmaf(th[L::oW2 + j * HID + i], h1[i], a);
        h2[j] = tanhf(a);
    }
#pragma unroll
    for (int j = 0; j < L::PP; ++j) {
        float a = th[L::ob3 + j] + omega * X[j];
#pragma unroll
        for (int i = 0; i < HID; ++i) a = fmaf(th[L::oW3 + j * HID + i], h2[i], a);
        y[j] = a;
    }
}

// D_e^-1 (or its transpose) times v, the inverse block packed in groups of 4 floats
template <int P, bool TRANS>
__device__ __forceinline__ void dinv_apply(const float *__restrict__ Dinv, int e, size_t NF, const float (&v)[P + 1],
                                           float (&out)[P + 1]) {
    constexpr int PP = P + 1;
#pragma unroll
    for (int r = 0; r < PP; ++r) out[r] = 0.f;
#pragma unroll
    for (int r = 0; r < PP; ++r)
#pragma unroll
        for (int c = 0; c < PP; ++c) {
            const int j = r * PP + c;
            const float d = __ldg(Dinv + packed_index(j, e, NF, 4));
            if (TRANS) out[c] = fmaf(d, v[r], out[c]);
            else out[r] = fmaf(d, v[c], out[r]);
        }
}

// x_out = x + c(r): the learned sweep
template <int P, int HID>
__global__ void __launch_bounds__(128) infer_kernel(int NF, const int32_t *__restrict__ nbr,
                                                    const float *__restrict__ r, const float *__restrict__ Dinv,
                                                    const float *__restrict__ theta, float omega,
                                                    const float *__restrict__ x, float *__restrict__ xout) {
    using L = LN<P, HID>;
    __shared__ float th[L::NPAR];
    for (int i = threadIdx.x; i < L::NPAR; i += blockDim.x) th[i] = theta[i];
    __syncthreads();
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NF) return;
    float X[L::F], h1[HID], h2[HID], y[L::PP], c[L::PP];
    const float s = patch_features<P>(nbr, r, e, NF, X);
    mlp<P, HID>(th, X, omega, h1, h2, y);
#pragma unroll
    for (int j = 0; j < L::PP; ++j) y[j] *= s;
    dinv_apply<P, false>(Dinv, e, NF, y, c);
#pragma unroll
    for (int j = 0; j < L::PP; ++j) xout[size_t(j) * NF + e] = x[size_t(j) * NF + e] + c[j];
}

// ---------------------------------------------------------------- tensor cores
// The same network on the 5th-generation tensor cores: the three layers are
// GEMMs of a tile of 128 facets (rows) against weights shared by all facets,
// BF16 operands in shared memory, FP32 accumulators in tensor memory,
//   H1 = tanh(X W1^T + b1),  H2 = tanh(H1 W2^T + b2),  Y = H2 W3^T + b3,
// one tcgen05.mma per 16-wide K step issued by one thread, completion signalled
// on an mbarrier (bounded wait).  The damped block-Jacobi part omega X_self,
// the scale s and the D^-1 solve stay FP32, so only the learned correction
// passes through BF16.  Operands use the canonical no-swizzle K-major layout:
// 8-row x 16-byte core matrices, element (row, k) at byte
//   (row / 8) * (K / 8) * 128 + (k / 8) * 128 + (row % 8) * 16 + (k % 8) * 2,
// i.e. leading (K-direction) core stride 128 B, stride (row-group) K / 8 * 128 B.
template <int P>
struct TC {
    static constexpr int PP = P + 1, F = 5 * PP, K1 = (F + 15) / 16 * 16, N3 = 16;
};

__device__ __forceinline__ int canon(int row, int k, int K) {
    return (row / 8) * (K / 8) * 64 + (k / 8) * 64 + (row % 8) * 8 + (k % 8);   // in bf16 elements
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor (no swizzle, K-major): start, leading and
// stride byte offsets (>> 4), descriptor version 1
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t K) {
    uint64_t d = uint64_t((addr & 0x3FFFF) >> 4);
    d |= uint64_t(128 >> 4) << 16;
    d |= uint64_t(((K / 8) * 128) >> 4) << 32;
    d |= uint64_t(1) << 46;
    return d;
}

// instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

// D (tensor memory) = sum over K steps of A (128 x K) B^T (N x K)
__device__ __forceinline__ void umma_gemm(uint32_t tmem, const void *A, const void *B, int K, uint32_t idesc) {
    for (int ks = 0; ks < K / 16; ++ks) {
        const uint64_t ad = umma_desc(smem_addr(A) + ks * 256, K), bd = umma_desc(smem_addr(B) + ks * 256, K);
        const uint32_t acc = ks > 0 ? 1u : 0u;
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                     :: "r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
    }
}

// thread 0: commit the issued MMAs to the barrier and wait (bounded) for the
// given phase; the outcome is published to the CTA
__device__ __forceinline__ bool umma_wait(uint64_t *bar, uint32_t phase, int *flag, int32_t *status) {
    if (threadIdx.x == 0) {
        int ok = 0;
        for (long long it = 0; it < (1ll << 24) && !ok; ++it) {
            uint32_t d;
            asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                         "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(d) : "r"(smem_addr(bar)), "r"(phase) : "memory");
            ok = int(d);
        }
        if (!ok) {
            // record it and give the MMAs one more bounded wait before the
            // tensor memory they write is freed
            atomicOr(status, 16);
            for (long long it = 0; it < (1ll << 24); ++it) {
                uint32_t d;
                asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                             "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(d) : "r"(smem_addr(bar)), "r"(phase) : "memory");
                if (d) break;
            }
        }
        *flag = ok;
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return *flag != 0;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr) : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// the hardware tanh approximation (about 11 significant bits): its result is
// rounded to BF16 (8 bits) right after
__device__ __forceinline__ float tanh_hw(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// own row of a layer: tanh(acc + bias) in BF16, written in the canonical layout
template <int HID>
__device__ __forceinline__ void hidden_epilogue(uint32_t tmem_row, const float *bias, __nv_bfloat16 *sH) {
    const int row = threadIdx.x;
#pragma unroll
    for (int c0 = 0; c0 < HID; c0 += 16) {
        float v[16];
        tmem_ld16(tmem_row + uint32_t(c0), v);
#pragma unroll
        for (int g = 0; g < 16; g += 8) {
            __align__(16) __nv_bfloat16 h8[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) h8[t] = __float2bfloat16_rn(tanh_hw(v[g + t] + bias[c0 + g + t]));
            *reinterpret_cast<uint4 *>(sH + canon(row, c0 + g, HID)) = *reinterpret_cast<const uint4 *>(h8);
        }
    }
}

// x_out = x + c(r) for 128 facets per CTA
template <int P, int HID>
__global__ void __launch_bounds__(128) infer_tc_kernel(int NF, const int32_t *__restrict__ nbr,
                                                       const float *__restrict__ r, const float *__restrict__ Dinv,
                                                       const float *__restrict__ theta,
                                                       const __nv_bfloat16 *__restrict__ wimg, float omega,
                                                       const float *__restrict__ x, float *__restrict__ xout,
                                                       int32_t *status) {
    using L = LN<P, HID>;
    using T = TC<P>;
    constexpr int PP = T::PP, F = T::F, K1 = T::K1, N3 = T::N3;
    constexpr int NW1 = HID * K1, NW2 = HID * HID, NW3 = N3 * HID;
    __shared__ __align__(128) __nv_bfloat16 sX[128 * K1];
    __shared__ __align__(128) __nv_bfloat16 sH[128 * HID];
    __shared__ __align__(128) __nv_bfloat16 sW[NW1 + NW2 + NW3];
    __shared__ float sb[2 * HID + PP];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    __shared__ int flag;
    const int tid = threadIdx.x, warp = tid / 32;
    const int e = blockIdx.x * 128 + tid;
    const bool valid = e < NF;
    // weights (BF16 images, canonical layout) and biases
    for (int i = tid; i < (NW1 + NW2 + NW3) / 8; i += 128)
        reinterpret_cast<uint4 *>(sW)[i] = reinterpret_cast<const uint4 *>(wimg)[i];
    for (int i = tid; i < HID; i += 128) {
        sb[i] = theta[L::ob1 + i];
        sb[HID + i] = theta[L::ob2 + i];
    }
    if (tid < PP) sb[2 * HID + tid] = theta[L::ob3 + tid];
    // features of the own facet (FP32), rounded to BF16 for the first GEMM
    float X[F];
    float s = 1.f;
    if (valid) {
        s = patch_features<P>(nbr, r, e, NF, X);
    } else {
#pragma unroll
        for (int i = 0; i < F; ++i) X[i] = 0.f;
    }
#pragma unroll
    for (int k0 = 0; k0 < K1; k0 += 8) {
        __align__(16) __nv_bfloat16 x8[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) x8[t] = __float2bfloat16_rn(k0 + t < F ? X[k0 + t] : 0.f);
        *reinterpret_cast<uint4 *>(sX + canon(tid, k0, K1)) = *reinterpret_cast<const uint4 *>(x8);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_addr(&tmem_base)), "r"(HID) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t tmem_row = tmem + (uint32_t(warp * 32) << 16);
    bool ok = true;
    // layer 1
    if (tid == 0) {
        umma_gemm(tmem, sX, sW, K1, umma_idesc(128, HID));
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(smem_addr(&bar)) : "memory");
    }
    ok = umma_wait(&bar, 0, &flag, status);
    if (ok) hidden_epilogue<HID>(tmem_row, sb, sH);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // layer 2 (same tensor-memory columns, read above)
    if (ok) {
        if (tid == 0) {
            umma_gemm(tmem, sH, sW + NW1, HID, umma_idesc(128, HID));
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_addr(&bar)) : "memory");
        }
        ok = umma_wait(&bar, 1, &flag, status);
        if (ok) hidden_epilogue<HID>(tmem_row, sb + HID, sH);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // layer 3 and the FP32 output
    if (ok) {
        if (tid == 0) {
            umma_gemm(tmem, sH, sW + NW1 + NW2, HID, umma_idesc(128, N3));
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_addr(&bar)) : "memory");
        }
        ok = umma_wait(&bar, 0, &flag, status);
        if (ok) {
            float acc[16];
            tmem_ld16(tmem_row, acc);
            if (valid) {
                float y[PP], c[PP];
#pragma unroll
                for (int j = 0; j < PP; ++j) y[j] = (acc[j] + sb[2 * HID + j] + omega * X[j]) * s;
                dinv_apply<P, false>(Dinv, e, NF, y, c);
#pragma unroll
                for (int j = 0; j < PP; ++j) xout[size_t(j) * NF + e] = x[size_t(j) * NF + e] + c[j];
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(HID) : "memory");
}

// theta -> BF16 images of W1, W2, W3 in the canonical layout (zero padding)
template <int P, int HID>
__global__ void tc_weights_kernel(const float *__restrict__ theta, __nv_bfloat16 *__restrict__ img) {
    using L = LN<P, HID>;
    using T = TC<P>;
    constexpr int F = T::F, K1 = T::K1, N3 = T::N3, PP = T::PP;
    constexpr int NW1 = HID * K1, NW2 = HID * HID, NW3 = N3 * HID;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < NW1) {
        const int j = i / K1, k = i % K1;
        img[canon(j, k, K1)] = __float2bfloat16_rn(k < F ? theta[L::oW1 + j * F + k] : 0.f);
    } else if (i < NW1 + NW2) {
        const int q = i - NW1, j = q / HID, k = q % HID;
        img[NW1 + canon(j, k, HID)] = __float2bfloat16_rn(theta[L::oW2 + j * HID + k]);
    } else if (i < NW1 + NW2 + NW3) {
        const int q = i - NW1 - NW2, j = q / HID, k = q % HID;
        img[NW1 + NW2 + canon(j, k, HID)] = __float2bfloat16_rn(j < PP ? theta[L::oW3 + j * HID + k] : 0.f);
    }
}

// training forward for one residual: c (internal layout) and the per-facet
// activations kept for the backward pass: act[e] = X (F) | h1 (HID) | h2 (HID) | s
template <int P, int HID>
__global__ void __launch_bounds__(128) train_forward_kernel(int NF, const int32_t *__restrict__ nbr,
                                                            const float *__restrict__ r, const float *__restrict__ Dinv,
                                                            const float *__restrict__ theta, float omega,
                                                            float *__restrict__ c_out, float *__restrict__ act) {
    using L = LN<P, HID>;
    constexpr int NA = L::F + 2 * HID + 1;
    __shared__ float th[L::NPAR];
    for (int i = threadIdx.x; i < L::NPAR; i += blockDim.x) th[i] = theta[i];
    __syncthreads();
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NF) return;
    float X[L::F], h1[HID], h2[HID], y[L::PP], c[L::PP];
    const float s = patch_features<P>(nbr, r, e, NF, X);
    mlp<P, HID>(th, X, omega, h1, h2, y);
    float *a = act + size_t(e) * NA;
#pragma unroll
    for (int i = 0; i < L::F; ++i) a[i] = X[i];
#pragma unroll
    for (int i = 0; i < HID; ++i) { a[L::F + i] = h1[i]; a[L::F + HID + i] = h2[i]; }
    a[NA - 1] = s;
#pragma unroll
    for (int j = 0; j < L::PP; ++j) y[j] *= s;
    dinv_apply<P, false>(Dinv, e, NF, y, c);
#pragma unroll
    for (int j = 0; j < L::PP; ++j) c_out[size_t(j) * NF + e] = c[j];
}

// y = S^T x with the packed FP32 facet-row operator: facet e collects its own
// diagonal block and, from each neighbour f, the block of f's row that
// multiplies e (rev[k][e] = f * 8 + block index)
template <int P>
__global__ void applyT_kernel(int NF, const float *__restrict__ Sval, const int32_t *__restrict__ rev,
                              const float *__restrict__ x, float *__restrict__ y) {
    constexpr int PP = P + 1;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NF) return;
    float acc[PP];
#pragma unroll
    for (int c = 0; c < PP; ++c) acc[c] = 0.f;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        int f = e, b = 0;
        if (k > 0) {
            const int code = rev[size_t(k - 1) * NF + e];
            f = code >> 3;
            b = code & 7;
        }
#pragma unroll
        for (int r = 0; r < PP; ++r) {
            const float xr = x[size_t(r) * NF + f];
#pragma unroll
            for (int c = 0; c < PP; ++c)
                acc[c] = fmaf(__ldg(Sval + packed_index((r * 5 + b) * PP + c, f, NF, 4)), xr, acc[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < PP; ++c) y[size_t(c) * NF + e] = acc[c];
}

// backward per facet: from gc = dL/dc (scaled by coef) to the per-facet
// gradients g = [ga1 (HID) | ga2 (HID) | gy (PP)] used by the reductions
template <int P, int HID>
__global__ void __launch_bounds__(128) train_backward_kernel(int NF, const float *__restrict__ gc,
                                                             const float *__restrict__ Dinv,
                                                             const float *__restrict__ theta,
                                                             const float *__restrict__ act, const double *coef,
                                                             float *__restrict__ gout) {
    using L = LN<P, HID>;
    constexpr int NA = L::F + 2 * HID + 1, NG = 2 * HID + L::PP;
    __shared__ float th[L::NPAR];
    for (int i = threadIdx.x; i < L::NPAR; i += blockDim.x) th[i] = theta[i];
    __syncthreads();
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NF) return;
    const float cf = float(coef[0]);
    const float *a = act + size_t(e) * NA;
    const float s = a[NA - 1];
    float g[L::PP], gy[L::PP];
#pragma unroll
    for (int j = 0; j < L::PP; ++j) g[j] = cf * gc[size_t(j) * NF + e];
    dinv_apply<P, true>(Dinv, e, NF, g, gy);
#pragma unroll
    for (int j = 0; j < L::PP; ++j) gy[j] *= s;
    float ga2[HID], ga1[HID];
#pragma unroll 4
    for (int i = 0; i < HID; ++i) {
        float v = 0.f;
#pragma unroll
        for (int j = 0; j < L::PP; ++j) v = fmaf(th[L::oW3 + j * HID + i], gy[j], v);
        const float h2 = a[L::F + HID + i];
        ga2[i] = v * (1.f - h2 * h2);
    }
#pragma unroll 4
    for (int i = 0; i < HID; ++i) {
        float v = 0.f;
#pragma unroll
        for (int j = 0; j < HID; ++j) v = fmaf(th[L::oW2 + j * HID + i], ga2[j], v);
        const float h1 = a[L::F + i];
        ga1[i] = v * (1.f - h1 * h1);
    }
    float *go = gout + size_t(e) * NG;
#pragma unroll
    for (int i = 0; i < HID; ++i) { go[i] = ga1[i]; go[HID + i] = ga2[i]; }
#pragma unroll
    for (int j = 0; j < L::PP; ++j) go[2 * HID + j] = gy[j];
}

// Weight gradients: every parameter is a sum over facets of a gradient column
// (gfac = [ga1 | ga2 | gy], NG per facet) times an activation column (act =
// [X | h1 | h2 | s], NA per facet) or 1 for a bias.  A block takes kGradChunk
// facets, staged 32 rows at a time in shared memory (coalesced rows); each
// thread accumulates its parameters (tid, tid + 256, ...) and writes one
// partial per parameter; grad_reduce_kernel adds the partials in block order.
constexpr int kGradChunk = 1024, kGradRows = 32, kGradMaxPer = 25;   // 256 x 25 >= 6149 (p = 4, hidden 64)

__device__ __forceinline__ void grad_param_cols(int idx, int hid, int F, int pp, int &q, int &a) {
    const int n1 = hid * F, n2 = n1 + hid, n3 = n2 + hid * hid, n4 = n3 + hid, n5 = n4 + pp * hid;
    if (idx < n1) { q = idx / F; a = idx % F; }
    else if (idx < n2) { q = idx - n1; a = -1; }
    else if (idx < n3) { q = hid + (idx - n2) / hid; a = F + (idx - n2) % hid; }
    else if (idx < n4) { q = hid + (idx - n3); a = -1; }
    else if (idx < n5) { q = 2 * hid + (idx - n4) / hid; a = F + hid + (idx - n4) % hid; }
    else { q = 2 * hid + (idx - n5); a = -1; }
}

__global__ void __launch_bounds__(256) grad_partial_kernel(int NF, int hid, int F, int pp, int npar,
                                                           const float *__restrict__ gfac,
                                                           const float *__restrict__ act,
                                                           float *__restrict__ partial) {
    extern __shared__ float sm[];
    const int NG = 2 * hid + pp, NA = F + 2 * hid + 1;
    float *sG = sm, *sA = sm + kGradRows * NG;
    float acc[kGradMaxPer];
    int qc[kGradMaxPer], ac[kGradMaxPer];
#pragma unroll
    for (int t = 0; t < kGradMaxPer; ++t) {
        acc[t] = 0.f;
        const int idx = threadIdx.x + t * blockDim.x;
        qc[t] = 0;
        ac[t] = -1;
        if (idx < npar) grad_param_cols(idx, hid, F, pp, qc[t], ac[t]);
    }
    const int e0 = blockIdx.x * kGradChunk, e1 = min(NF, e0 + kGradChunk);
    for (int eb = e0; eb < e1; eb += kGradRows) {
        const int nr = min(kGradRows, e1 - eb);
        for (int i = threadIdx.x; i < nr * NG; i += blockDim.x) sG[i] = gfac[size_t(eb) * NG + i];
        for (int i = threadIdx.x; i < nr * NA; i += blockDim.x) sA[i] = act[size_t(eb) * NA + i];
        __syncthreads();
#pragma unroll
        for (int t = 0; t < kGradMaxPer; ++t) {
            if (threadIdx.x + t * blockDim.x < npar) {
                float v = acc[t];
                for (int r = 0; r < nr; ++r)
                    v = fmaf(sG[r * NG + qc[t]], ac[t] >= 0 ? sA[r * NA + ac[t]] : 1.f, v);
                acc[t] = v;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int t = 0; t < kGradMaxPer; ++t) {
        const int idx = threadIdx.x + t * blockDim.x;
        if (idx < npar) partial[size_t(blockIdx.x) * npar + idx] = acc[t];
    }
}

__global__ void grad_reduce_kernel(int nblk, int npar, const float *__restrict__ partial, float *__restrict__ grad) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= npar) return;
    float v = 0.f;
    for (int b = 0; b < nblk; ++b) v += partial[size_t(b) * npar + idx];
    grad[idx] += v;
}

__global__ void adam_kernel(int n, float *__restrict__ theta, float *__restrict__ m, float *__restrict__ v,
                            const float *__restrict__ g, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

#define HDG_LN_DISPATCH(p, hid, CALL)                                                          \
    switch ((p) * 100 + (hid)) {                                                                \
        case 132: { constexpr int P = 1, HID = 32; CALL; } break;                               \
        case 232: { constexpr int P = 2, HID = 32; CALL; } break;                               \
        case 332: { constexpr int P = 3, HID = 32; CALL; } break;                               \
        case 432: { constexpr int P = 4, HID = 32; CALL; } break;                               \
        case 164: { constexpr int P = 1, HID = 64; CALL; } break;                               \
        case 264: { constexpr int P = 2, HID = 64; CALL; } break;                               \
        case 364: { constexpr int P = 3, HID = 64; CALL; } break;                               \
        case 464: { constexpr int P = 4, HID = 64; CALL; } break;                               \
        default: return cudaErrorInvalidValue;                                                  \
    }

// dst = src / sqrt(nrm2[0])
__global__ void normalize_kernel(const float *src, float *dst, const double *nrm2, size_t n) {
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = float(double(src[i]) / sqrt(nrm2[0]));
}

// [NF][PP] -> [PP][NF] for FP32 vectors
__global__ void to_internal32_kernel(int NF, int PP, const float *ext, float *in) {
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= size_t(NF) * PP) return;
    in[(i % PP) * NF + i / PP] = ext[i];
}

// [PP][NF] -> [NF][PP] for FP32 vectors
__global__ void to_external32_kernel(int NF, int PP, const float *in, float *ext) {
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= size_t(NF) * PP) return;
    ext[i] = in[(i % PP) * NF + i / PP];
}

}  // namespace

cudaError_t launch_to_external32(hdg_handle *h, const float *in, float *ext) {
    const size_t n = size_t(h->NF) * h->pp;
    to_external32_kernel<<<blocks(n, 256), 256, 0, h->stream>>>(h->NF, h->pp, in, ext);
    return cudaGetLastError();
}

cudaError_t launch_normalize32(const float *src, float *dst, const double *nrm2, size_t n, cudaStream_t s) {
    normalize_kernel<<<blocks(n, 256), 256, 0, s>>>(src, dst, nrm2, n);
    return cudaGetLastError();
}
cudaError_t launch_to_internal32(hdg_handle *h, const float *ext, float *in) {
    const size_t n = size_t(h->NF) * h->pp;
    to_internal32_kernel<<<blocks(n, 256), 256, 0, h->stream>>>(h->NF, h->pp, ext, in);
    return cudaGetLastError();
}

int learned_n_params(int p, int hid) {
    const int pp = p + 1, F = 5 * pp;
    return hid * F + hid + hid * hid + hid + pp * hid + pp;
}

cudaError_t launch_learned_infer(hdg_handle *h, const float *r, const float *x, float *xout) {
    HDG_LN_DISPATCH(h->p, h->lc.hid,
                    (infer_kernel<P, HID><<<blocks(h->NF, 128), 128, 0, h->stream>>>(h->NF, h->d_nbr, r, h->d_Dinv32,
                                                                                      h->lc.theta, float(h->prm.omega), x,
                                                                                      xout)));
    return cudaGetLastError();
}

cudaError_t launch_learned_infer_tc(hdg_handle *h, const float *r, const float *x, float *xout) {
    HDG_LN_DISPATCH(h->p, h->lc.hid,
                    (infer_tc_kernel<P, HID><<<blocks(h->NF, 128), 128, 0, h->stream>>>(
                        h->NF, h->d_nbr, r, h->d_Dinv32, h->lc.theta, h->lc.wimg, float(h->prm.omega), x, xout,
                        h->d_status)));
    return cudaGetLastError();
}

size_t learned_tc_image_elems(int p, int hid) {
    const int F = 5 * (p + 1), K1 = (F + 15) / 16 * 16;
    return size_t(hid) * K1 + size_t(hid) * hid + size_t(16) * hid;
}

cudaError_t launch_learned_tc_weights(hdg_handle *h) {
    const size_t n = learned_tc_image_elems(h->p, h->lc.hid);
    HDG_LN_DISPATCH(h->p, h->lc.hid,
                    (tc_weights_kernel<P, HID><<<blocks(n, 256), 256, 0, h->stream>>>(h->lc.theta, h->lc.wimg)));
    return cudaGetLastError();
}

// one training pass over residual r: adds its gradient (times coef) to lc.grad
cudaError_t launch_learned_forward(hdg_handle *h, const float *r, float *c) {
    HDG_LN_DISPATCH(h->p, h->lc.hid,
                    (train_forward_kernel<P, HID><<<blocks(h->NF, 128), 128, 0, h->stream>>>(
                        h->NF, h->d_nbr, r, h->d_Dinv32, h->lc.theta, float(h->prm.omega), c, h->lc.act)));
    return cudaGetLastError();
}

cudaError_t launch_learned_applyT(hdg_handle *h, const float *x, float *y) {
    switch (h->p) {
        case 1: applyT_kernel<1><<<blocks(h->NF, 256), 256, 0, h->stream>>>(h->NF, h->d_Sval32, h->lc.rev, x, y); break;
        case 2: applyT_kernel<2><<<blocks(h->NF, 256), 256, 0, h->stream>>>(h->NF, h->d_Sval32, h->lc.rev, x, y); break;
        case 3: applyT_kernel<3><<<blocks(h->NF, 256), 256, 0, h->stream>>>(h->NF, h->d_Sval32, h->lc.rev, x, y); break;
        case 4: applyT_kernel<4><<<blocks(h->NF, 256), 256, 0, h->stream>>>(h->NF, h->d_Sval32, h->lc.rev, x, y); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_learned_backward(hdg_handle *h, const float *gc, const double *coef) {
    const int hid = h->lc.hid, pp = h->pp, F = 5 * pp;
    HDG_LN_DISPATCH(h->p, hid,
                    (train_backward_kernel<P, HID><<<blocks(h->NF, 128), 128, 0, h->stream>>>(
                        h->NF, gc, h->d_Dinv32, h->lc.theta, h->lc.act, coef, h->lc.gfac)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int NA = F + 2 * hid + 1, NG = 2 * hid + pp;
    // dW1 = ga1 X^T, db1 = sum ga1; dW2 = ga2 h1^T, db2; dW3 = gy h2^T, db3
    const int npar = h->lc.npar;
    if (npar > 256 * kGradMaxPer) return cudaErrorInvalidValue;
    const int nblk = int((h->NF + kGradChunk - 1) / kGradChunk);
    const size_t smem = sizeof(float) * kGradRows * size_t(NG + NA);
    grad_partial_kernel<<<nblk, 256, smem, h->stream>>>(int(h->NF), hid, F, pp, npar, h->lc.gfac, h->lc.act,
                                                         h->lc.gpart);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    grad_reduce_kernel<<<blocks(npar, 256), 256, 0, h->stream>>>(nblk, npar, h->lc.gpart, h->lc.grad);
    return cudaGetLastError();
}

cudaError_t launch_adam(hdg_handle *h, float lr, int t) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, float(t)), c2 = 1.f - powf(b2, float(t));
    const int n = h->lc.npar;
    adam_kernel<<<blocks(n, 256), 256, 0, h->stream>>>(n, h->lc.theta, h->lc.m, h->lc.v, h->lc.grad, lr, b1, b2, 1e-8f,
                                                      c1, c2);
    return cudaGetLastError();
}

}  // namespace hdg
