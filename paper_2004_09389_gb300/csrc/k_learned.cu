// Learned facet-patch smoother (spec extension; the paper has none).
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

// grad[out_off + i * nb + j] += sum_e A[e][ao + i] * B[e][bo + j] (B = 1 when nb = 0: bias,
// written at out_off + i).  One block per i, threads over facets, fixed-order
// tree reduction per j: deterministic.
__global__ void outer_reduce_kernel(int NF, const float *__restrict__ A, int lda, int ao,
                                    const float *__restrict__ Bm, int ldb, int bo, int nb, float *__restrict__ grad,
                                    int out_off) {
    __shared__ float red[256];
    const int i = blockIdx.x;
    const int ncol = nb > 0 ? nb : 1;
    for (int j = 0; j < ncol; ++j) {
        float acc = 0.f;
        for (int e = threadIdx.x; e < NF; e += blockDim.x) {
            const float av = A[size_t(e) * lda + ao + i];
            acc = fmaf(av, nb > 0 ? Bm[size_t(e) * ldb + bo + j] : 1.f, acc);
        }
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int sft = blockDim.x / 2; sft > 0; sft >>= 1) {
            if (threadIdx.x < sft) red[threadIdx.x] += red[threadIdx.x + sft];
            __syncthreads();
        }
        if (threadIdx.x == 0) grad[out_off + (nb > 0 ? i * nb + j : i)] += red[0];
        __syncthreads();
    }
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
__global__ void normalize_kernel(const float *__restrict__ src, float *__restrict__ dst, const double *nrm2, size_t n) {
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
    const int oW1 = 0, ob1 = hid * F, oW2 = ob1 + hid, ob2 = oW2 + hid * hid, oW3 = ob2 + hid, ob3 = oW3 + pp * hid;
    float *gr = h->lc.grad;
    // dW1 = ga1 X^T, db1 = sum ga1; dW2 = ga2 h1^T, db2; dW3 = gy h2^T, db3
    outer_reduce_kernel<<<hid, 256, 0, h->stream>>>(h->NF, h->lc.gfac, NG, 0, h->lc.act, NA, 0, F, gr, oW1);
    outer_reduce_kernel<<<hid, 256, 0, h->stream>>>(h->NF, h->lc.gfac, NG, 0, nullptr, 0, 0, 0, gr, ob1);
    outer_reduce_kernel<<<hid, 256, 0, h->stream>>>(h->NF, h->lc.gfac, NG, hid, h->lc.act, NA, F, hid, gr, oW2);
    outer_reduce_kernel<<<hid, 256, 0, h->stream>>>(h->NF, h->lc.gfac, NG, hid, nullptr, 0, 0, 0, gr, ob2);
    outer_reduce_kernel<<<pp, 256, 0, h->stream>>>(h->NF, h->lc.gfac, NG, 2 * hid, h->lc.act, NA, F + hid, hid, gr, oW3);
    outer_reduce_kernel<<<pp, 256, 0, h->stream>>>(h->NF, h->lc.gfac, NG, 2 * hid, nullptr, 0, 0, 0, gr, ob3);
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
