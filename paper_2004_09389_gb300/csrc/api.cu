// C ABI of the HDG trace solver: handle lifecycle, condensation, the
// two-level preconditioner, the Krylov drivers and the entry points of hdg.h.
//
// Solve (Sec. 4.2): step 1 builds g = sum_K P_K^T C_K A_K^-1 F_K; step 2 solves
// S lambda = g (Eq. schur_system) with right-preconditioned FGMRES whose
// preconditioner is one pass of Alg. twolevel_vcycle (zero initial guess):
// n_pre block-Jacobi sweeps, residual, restriction to P1 (pi^T), a geometric
// P1 V-cycle for the coarse problem of Eq. coarse_problem_upwind, prolongation
// (pi) and n_post sweeps.  Step 3 recovers (u, h) cell by cell.
// HDG_MIXED_FP32 runs step 2 as FP64 iterative refinement: the residual
// g - S lambda and the update of lambda are FP64, each correction comes from an
// FP32 FGMRES on the FP32 copy of the operator and preconditioner.
#include "common.h"

#include <algorithm>
#include <type_traits>
#include <atomic>
#include <thread>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>

#include <chrono>
#include <ucontext.h>

namespace hdg {

template <typename T> cudaError_t launch_apply_t(hdg_handle *, const T *, T *);
template <typename T> cudaError_t launch_residual_t(hdg_handle *, const T *, const T *, T *, bool);
template <typename T> cudaError_t launch_smooth_t(hdg_handle *, const T *, const T *, T *);
template <typename T>
cudaError_t launch_smooth_first_t(hdg_handle *, const T *, T *, const T * = nullptr, const double * = nullptr,
                                  T * = nullptr, double = 0.0);
template <typename T>
cudaError_t launch_smooth_cheb_t(hdg_handle *, const T *, const T *, T *, double, double, const T *);
template <typename T>
cudaError_t launch_apply_dots_t(hdg_handle *, const T *, T *, const T *, size_t, int, double *, unsigned int *,
                                double *);
template <typename T> cudaError_t launch_restrict_t(hdg_handle *, const T *, T *, const T *, T, T *);
template <typename T>
cudaError_t launch_smooth_prolong_t(hdg_handle *, const T *, const T *, const T *, T *, double = 0.0, T * = nullptr);
template <typename T> cudaError_t launch_prolong_add_t(hdg_handle *, const T *, T *);

// Krylov vectors of one precision
template <typename T>
struct KSpace {
    T *V = nullptr, *Z = nullptr, *w = nullptr;      // (m+1) x NT, m x NT, NT
    T *t0 = nullptr, *t1 = nullptr, *res = nullptr;  // preconditioner work
    T *b = nullptr, *x = nullptr;                    // right-hand side / solution (FP32 inner solve)
};

struct Workspace {
    int m = 0;
    size_t NT = 0;
    size_t ld = 0;        // leading dimension of the Krylov basis (NT rounded up to 16 bytes, zero padded)
    int nchunk = 1;
    int nblk_gs = 1;      // blocks of the fused Gram-Schmidt kernels
    unsigned int *counter = nullptr;
    ReadBack *rb = nullptr;
    // page-locked readbacks, one slot per Arnoldi step j (written by its
    // Gram-Schmidt kernel), their device address, and per slot whether a
    // launched step may still write it (set at launch, cleared once the host
    // has seen the step's number)
    ReadBack *host_rb = nullptr, *host_rb_dev = nullptr;
    std::vector<char> rb_pending;
    HostValue *host_val = nullptr, *host_val_dev = nullptr;   // norms handed to the host
    int32_t val_seq = 0;
    double *g = nullptr, *x = nullptr, *r = nullptr, *ycell = nullptr;
    float2 *x2 = nullptr;  // mixed modes: split copy of the FP64 iterate x (two-float residual)
    KSpace<double> k64;
    KSpace<float> k32;
    // small device arrays
    double *Hm = nullptr, *cs = nullptr, *sn = nullptr, *sv = nullptr, *h1 = nullptr, *h2 = nullptr;
    double *nrm2 = nullptr, *est = nullptr, *y = nullptr, *partial = nullptr;
    double *scal = nullptr;   // restart normalisation of a Krylov cycle
    double *bnorm = nullptr;  // ||b|| of the current Krylov solve
    // CUDA graphs of one Arnoldi step per (precision, j); see arnoldi_step
    struct StepGraph { cudaGraphExec_t exec = nullptr; int64_t counts[HDG_PROF_N] = {}; const void *src = nullptr; };
    // slots 0..m-1: step j; slot m: step 0 forming v_0 from the right-hand side (src)
    std::vector<StepGraph> graphs[3];   // FP64, FP32, FP32 with the learned sweep
    bool use_graphs = true;
    double *beta = nullptr;   // refinement scale ||g - S x|| (mixed mode)
    int32_t *flags = nullptr;
    // pinned readback
    double *host_buf = nullptr;   // [8]: 0 readback, 1 restart scale, 2 refinement scale, 3 s_0, 4 ||b||
    double *host_buf_dev = nullptr;   // its device address (read by recorded copies in batched solves)
    int32_t *host_flags = nullptr;
    // staging for host-pointer entry points and for recover defaults
    double *ru = nullptr, *rh = nullptr, *lam_ext = nullptr, *u = nullptr, *hh = nullptr;
    double *ru_x = nullptr, *rh_x = nullptr;   // explicit hdg_recover inputs (ru/rh keep the last solve's)
    bool have_rhs = false, have_lambda = false;
    // two-float handles: z_K = R_M r_K of the last solve's right-hand side ([nK][N]
    // pairs, written by its step 1), valid until the operator changes
    float2 *z2 = nullptr;
    bool have_z = false;
    double *lam_int = nullptr;    // last solution, internal layout
};

}  // namespace hdg

using namespace hdg;

namespace {

thread_local std::string g_setup_error;

int fail(hdg_handle *h, int code, const std::string &msg) {
    if (h) h->err = msg;
    else g_setup_error = msg;
    return code;
}

#define TRY(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return fail(h, HDG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// every device array is its own allocation, padded to a multiple of 16 bytes
// (TMA bulk copies move whole 16-byte words)
template <typename T>
cudaError_t dalloc(T **p, size_t n) {
    *p = nullptr;
    if (n == 0) return cudaSuccess;
    return cudaMalloc(reinterpret_cast<void **>(p), (n * sizeof(T) + 15) / 16 * 16);
}
template <typename T>
cudaError_t upload(T **p, const std::vector<T> &v, cudaStream_t s) {
    cudaError_t e = dalloc(p, v.size());
    if (e != cudaSuccess || v.empty()) return e;
    return cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s);
}
template <typename T>
void dfree(T *&p) {
    if (p) cudaFree(p);
    p = nullptr;
}

// Device address under which kernels may access a host buffer in place
// (page-locked memory from cudaHostAlloc / cudaHostRegister on this device;
// on Grace-Blackwell such accesses cross the coherent NVLink-C2C link), or
// nullptr for other memory, which goes through staged copies.  The caller's
// buffer must span the documented size, as for the copies.
template <typename T>
T *host_alias(T *p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    if (a.type != cudaMemoryTypeHost || !a.devicePointer || a.device != dev) return nullptr;
    return static_cast<T *>(a.devicePointer);
}

std::string check_params(const hdg_params *prm) {
    if (!prm) return "params is NULL";
    if (prm->p < 1 || prm->p > 4) return "p must be in 1..4";
    if (!(prm->tau > 0) || !(prm->g > 0) || !(prm->H > 0)) return "tau, g and H must be positive";
    if (!(prm->rtol > 0)) return "rtol must be positive";
    if (prm->restart < 1 || prm->restart > 64) return "restart must be in 1..64";
    if (prm->max_iter < 1) return "max_iter must be positive";
    if (prm->n_pre < 0 || prm->n_post < 0 || prm->p1_nu_pre < 0 || prm->p1_nu_post < 0) return "negative sweep count";
    if (!(prm->omega > 0) || !(prm->p1_omega > 0)) return "damping factors must be positive";
    if (prm->coarse_mode < 0 || prm->coarse_mode > 2) return "coarse_mode must be 0, 1 or 2";
    if (prm->reorth != 0 && prm->reorth != 1) return "reorth must be 0 or 1";
    if (prm->smoother != 0 && prm->smoother != 1) return "smoother must be 0 or 1";
    if (prm->flux != 0 && prm->flux != 1) return "flux must be 0 or 1";
    if (prm->keep_rhs != 0 && prm->keep_rhs != 1) return "keep_rhs must be 0 or 1";
    if (prm->flux == 1) {
        if (prm->precision != HDG_FP64) return "the Lax-Friedrichs solver runs in HDG_FP64";
        if (prm->p < 1 || prm->p > 2) return "the Lax-Friedrichs solver supports p = 1 and 2";
        if (prm->coarse_mode == 2) return "the Lax-Friedrichs solver uses coarse_mode 0 or 1";
        if (prm->n_coarse < 1 || prm->n_coarse > 200) return "n_coarse must be in 1..200";
        if (prm->cheb_steps < 2 || prm->cheb_steps > 64) return "cheb_steps must be in 2..64";
    }
    if (prm->smoother == 1 && prm->cheb_theta <= 0 && (prm->cheb_steps < 2 || prm->cheb_steps > 64))
        return "cheb_steps must be in 2..64";
    if (prm->smoother == 1 && prm->cheb_theta > 0 && !(std::isfinite(prm->cheb_delta2) &&
                                                       prm->cheb_delta2 < prm->cheb_theta * prm->cheb_theta))
        return "cheb_delta2 must be finite and below cheb_theta^2";
    if (prm->precision != HDG_FP64 && prm->precision != HDG_MIXED_FP32 && prm->precision != HDG_MIXED_BF16 &&
        prm->precision != HDG_MIXED_FGMRES64)
        return "unknown precision mode";
    if ((prm->precision == HDG_MIXED_FP32 || prm->precision == HDG_MIXED_BF16) &&
        !(prm->inner_rtol > 0 && prm->inner_rtol < 1))
        return "inner_rtol must be in (0, 1)";
    return "";
}

// ---------------------------------------------------------------- kernel accounting

cudaEvent_t prof_event(hdg_handle *h) {
    Prof &P = h->prof;
    if (!P.pool.empty()) {
        cudaEvent_t e = P.pool.back();
        P.pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Sum the elapsed times of the bracketed launches; call after a stream sync.
void prof_flush(hdg_handle *h) {
    Prof &P = h->prof;
    for (auto &q : P.pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) P.ms[q.cat] += ms;
        P.pool.push_back(q.a);
        P.pool.push_back(q.b);
    }
    P.pending.clear();
}

// Launch through f(), counting nk kernels in category cat and, with timing
// on, bracketing them with events on the handle's stream.
template <class F>
cudaError_t klaunch(hdg_handle *h, int cat, int nk, F &&f) {
    Prof &P = h->prof;
    P.launches[cat] += nk;
    if (!P.on) return f();
    cudaEvent_t a = prof_event(h), b = prof_event(h);
    if (P.evict_buf) launch_l2_evict(P.evict_buf, P.evict_bytes, P.evict_sink, h->stream);
    cudaEventRecord(a, h->stream);
    cudaError_t e = f();
    cudaEventRecord(b, h->stream);
    P.pending.push_back({cat, a, b});
    return e;
}
#define KL(cat, nk, expr) klaunch(h, (cat), (nk), [&]() { return (expr); })

}  // namespace

bool hdg::solve_kept_z(const hdg_handle *h) { return h && h->ws && h->ws->have_z; }

cudaError_t hdg::account_launch(hdg_handle *h, int cat, int nk, const std::function<cudaError_t()> &fn) {
    return klaunch(h, cat, nk, fn);
}

namespace {

template <typename T> constexpr int cat_apply() { return sizeof(T) == 8 ? HDG_PROF_APPLY64 : HDG_PROF_APPLY32; }
template <typename T> constexpr int cat_res() { return sizeof(T) == 8 ? HDG_PROF_RESIDUAL64 : HDG_PROF_RESIDUAL32; }
template <typename T> constexpr int cat_smooth() { return sizeof(T) == 8 ? HDG_PROF_SMOOTH64 : HDG_PROF_SMOOTH32; }
template <typename T> constexpr int cat_first() { return sizeof(T) == 8 ? HDG_PROF_SMOOTH_FIRST64 : HDG_PROF_SMOOTH_FIRST32; }

// Stream-ordered copy of bytes on the handle's stream.  Inside a batched
// solve it is recorded as a copy kernel; a host source (only the page-locked
// scalar buffer is used as one) is then read through its device address.
cudaError_t dcopy(hdg_handle *h, void *dst, const void *src, size_t bytes, cudaMemcpyKind kind) {
    if (batch_recorder()) {
        const Workspace &W = *h->ws;
        if (kind == cudaMemcpyHostToDevice) {
            const double *p = static_cast<const double *>(src);
            if (!(p >= W.host_buf && p < W.host_buf + 8)) return cudaErrorInvalidValue;
            src = W.host_buf_dev + (p - W.host_buf);
        }
        return launch_copy(dst, src, bytes, h->stream);
    }
    return cudaMemcpyAsync(dst, src, bytes, kind, h->stream);
}
// Stream-ordered zero fill (recorded inside a batched solve, as dcopy)
cudaError_t dzero(hdg_handle *h, void *dst, size_t bytes) {
    if (batch_recorder()) return launch_copy(dst, nullptr, bytes, h->stream);
    return cudaMemsetAsync(dst, 0, bytes, h->stream);
}

// Inside a batched solve: give control back to the batch until the word at
// addr (page-locked, written by a recorded kernel) holds want (defined with
// the batch entry points)
int batch_yield(hdg_handle *h, const volatile int32_t *addr, int32_t want);

// ---------------------------------------------------------------- preconditioner

template <typename T>
const T *levA(const DevLevel &L);
template <>
const double *levA<double>(const DevLevel &L) { return L.A; }
template <>
const float *levA<float>(const DevLevel &L) { return L.A32; }
template <typename T>
const T *levD(const DevLevel &L);
template <>
const double *levD<double>(const DevLevel &L) { return L.dinv; }
template <>
const float *levD<float>(const DevLevel &L) { return L.dinv32; }
template <typename T>
T *levX(DevLevel &L);
template <>
double *levX<double>(DevLevel &L) { return L.x; }
template <>
float *levX<float>(DevLevel &L) { return L.x32; }
template <typename T>
T *levX2(DevLevel &L);
template <>
double *levX2<double>(DevLevel &L) { return L.x2; }
template <>
float *levX2<float>(DevLevel &L) { return L.x232; }
template <typename T>
T *levB(DevLevel &L);
template <>
double *levB<double>(DevLevel &L) { return L.b; }
template <>
float *levB<float>(DevLevel &L) { return L.b32; }
template <typename T>
T *levR(DevLevel &L);
template <>
double *levR<double>(DevLevel &L) { return L.r; }
template <>
float *levR<float>(DevLevel &L) { return L.r32; }
template <typename T>
KSpace<T> &kspace(hdg_handle *h);
template <>
KSpace<double> &kspace<double>(hdg_handle *h) { return h->ws->k64; }
template <>
KSpace<float> &kspace<float>(hdg_handle *h) { return h->ws->k32; }

}  // namespace

// sizes of the single-CTA levels [first, lev.size()) for their layout
static std::vector<TailLevelSize> tail_sizes(const std::vector<DevLevel> &lev, int first) {
    std::vector<TailLevelSize> lv;
    for (size_t l = size_t(first); l < lev.size(); ++l) {
        const bool top = int(l) == first;
        lv.push_back({lev[l].nv, lev[l].nnz, lev[l].width, top ? 0 : lev[l].nci, top ? 0 : lev[l - 1].nv});
    }
    return lv;
}

size_t hdg::tail_smem_bytes(const std::vector<DevLevel> &lev, int first, size_t tsz) {
    TailLayout lay;
    tail_layout(tail_sizes(lev, first), tsz, 0, lay);
    return lay.smem_bytes;
}

namespace {

template <typename T>
cudaError_t dots(hdg_handle *h, const T *V, int k, const T *w, double *out, HostValue *pub = nullptr,
                 int32_t seq = 0, double *root_a = nullptr, double *root_b = nullptr);

// P1 V-cycle for the coarse problem (Eq. coarse_problem_upwind) with
// right-hand side levB(level 0).  Levels above the tail: the first
// pre-smoothing sweep of each level rides on the restriction that produced
// its right-hand side; on levels with patches (at most 32,768 vertices) the
// last pre-sweep, the residual and the restriction share one patch kernel, and
// so do the prolongation and the first two post-sweeps; elsewhere one kernel
// per sweep, with the residual inside the restriction and the prolongation
// inside the first post-sweep.  Levels from tail_start down: one single-CTA
// kernel.  Returns the device vector that holds the level-0 result.  The first
// pre-smoothing sweep of level 0 (when it is above the tail) was done by the
// trace-to-P1 restriction.
template <typename T>
cudaError_t p1_cycle(hdg_handle *h, T **result) {
    cudaStream_t s = h->stream;
    const int nlev = int(h->lev.size()), ts = h->tail_start[sizeof(T) == 8 ? 0 : 1];
    const int nu1 = h->prm.p1_nu_pre, nu2 = h->prm.p1_nu_post;
    const T om = T(h->prm.p1_omega);
    std::vector<T *> cur(nlev), oth(nlev), res(nlev);
    cudaError_t e;
    for (int l = 0; l < ts; ++l) {
        DevLevel &L = h->lev[l];
        T *x = levX<T>(L), *x2 = levX2<T>(L);
        DevLevel &C = h->lev[l + 1];
        const bool fuse = (l + 1 < ts) && nu1 >= 1;
        // with two or more sweeps, the last one shares the patch kernel of the restriction
        const bool patch = h->p1_fused && p1_patch_ok<T>(L) && nu1 >= 2;
        if (nu1 == 0 && (e = KL(HDG_PROF_P1, 1, launch_fill<T>(x, T(0), L.nv, s))) != cudaSuccess) return e;
        for (int k = patch ? 2 : 1; k < nu1; ++k) {
            if ((e = KL(HDG_PROF_P1, 1, launch_p1_jacobi<T>(L, levA<T>(L), levD<T>(L), levB<T>(L), x, x2, om, false, s))) != cudaSuccess) return e;
            std::swap(x, x2);
        }
        if (patch) {
            if ((e = KL(HDG_PROF_P1, 1, launch_p1_down_fused<T>(L, C, levA<T>(L), levD<T>(L), levB<T>(L), x, x2,
                                                                levD<T>(C), om, levB<T>(C),
                                                                fuse ? levX<T>(C) : nullptr, s))) != cudaSuccess) return e;
            std::swap(x, x2);
        } else {
            if ((e = KL(HDG_PROF_P1, 1, launch_p1_down<T>(L, C, levA<T>(L), levB<T>(L), x, levD<T>(C), om, levB<T>(C),
                                                          fuse ? levX<T>(C) : nullptr, s))) != cudaSuccess) return e;
        }
        cur[l] = x; oth[l] = x2;
    }
    if (nlev - ts == 1 && h->lev[ts].nv > kTailDenseMax) {
        // the coarsest level alone, too large for one CTA's dense product: the
        // exact solve as a product with its FP64 inverse over many CTAs
        if ((e = KL(HDG_PROF_P1, 1, launch_p1_coarse_dense<T>(h->d_coarse_inv, h->lev[ts].nv, levB<T>(h->lev[ts]),
                                                               levX<T>(h->lev[ts]), s))) != cudaSuccess)
            return e;
        res[ts] = levX<T>(h->lev[ts]);
    } else {
        const TailImage &im = h->tail_img[sizeof(T) == 8 ? 0 : 1];
        if (im.ts != ts || !im.d) return cudaErrorInvalidValue;   // image not built for this tail start
        TailArgs a{};
        a.nlev = nlev - ts;
        a.nu1 = nu1;
        a.nu2 = nu2;
        a.omega = h->prm.p1_omega;
        a.img = im.d;
        a.img_bytes = im.img_bytes;
        a.inv_off = im.inv_off;
        a.nv0 = h->lev[ts].nv;
        a.ob0 = im.ob0;
        a.ox0 = im.ox0;
        a.dinv0 = levD<T>(h->lev[ts]);
        a.inv = h->d_coarse_inv;          // the coarsest solve stays FP64 in every precision
        a.status = h->d_status;
        a.b_top = levB<T>(h->lev[ts]);
        a.x_top = levX<T>(h->lev[ts]);
        const size_t smem = im.smem_bytes;
        if ((e = KL(HDG_PROF_P1, 1, launch_p1_tail<T>(a, smem, s))) != cudaSuccess) return e;
        res[ts] = levX<T>(h->lev[ts]);
    }
    for (int l = ts - 1; l >= 0; --l) {
        DevLevel &L = h->lev[l];
        DevLevel &C = h->lev[l + 1];
        T *x = cur[l], *x2 = oth[l];
        if (nu2 == 0) {
            if ((e = KL(HDG_PROF_P1, 1, launch_p1_prolong_add<T>(C, L.nv, res[l + 1], x, s))) != cudaSuccess) return e;
        } else if (h->p1_fused && p1_patch_ok<T>(L) && nu2 >= 2) {
            // the prolongation and the first two post-smoothing sweeps in one patch kernel
            if ((e = KL(HDG_PROF_P1, 1, launch_p1_up_fused<T>(L, C, levA<T>(L), levD<T>(L), levB<T>(L), x, res[l + 1], x2, om, s))) != cudaSuccess) return e;
            std::swap(x, x2);
            for (int k = 2; k < nu2; ++k) {
                if ((e = KL(HDG_PROF_P1, 1, launch_p1_jacobi<T>(L, levA<T>(L), levD<T>(L), levB<T>(L), x, x2, om, false, s))) != cudaSuccess) return e;
                std::swap(x, x2);
            }
        } else {
            if ((e = KL(HDG_PROF_P1, 1, launch_p1_up<T>(L, C, levA<T>(L), levD<T>(L), levB<T>(L), x, res[l + 1], x2, om, s))) != cudaSuccess) return e;
            std::swap(x, x2);
            for (int k = 1; k < nu2; ++k) {
                if ((e = KL(HDG_PROF_P1, 1, launch_p1_jacobi<T>(L, levA<T>(L), levD<T>(L), levB<T>(L), x, x2, om, false, s))) != cudaSuccess) return e;
                std::swap(x, x2);
            }
        }
        res[l] = x;
    }
    *result = res[0];
    return cudaSuccess;
}

// z = V(v), Alg. twolevel_vcycle with zero initial guess (internal layout).
// The same algorithm for the Lax-Friedrichs trace system (FP64): block-Jacobi
// or Chebyshev smoothing on the 2(p+1) x 2(p+1) facet blocks, restriction
// pi^T to RT0, n_coarse Chebyshev steps on the RT0 coarse problem from zero,
// x += pi e_c, post-smoothing.
cudaError_t precond_lf(hdg_handle *h, const double *v, double *z, const double *w_src) {
    KSpace<double> &k = h->ws->k64;
    cudaStream_t s = h->stream;
    const size_t NT = h->NT;
    const bool cheb = h->prm.smoother == 1;
    double *x = k.t0, *x2 = k.t1;
    cudaError_t e;
    // pre-smoothing from zero
    if (h->prm.n_pre == 0) {
        if ((e = KL(HDG_PROF_KRYLOV, 1, launch_fill<double>(x, 0.0, NT, s))) != cudaSuccess) return e;
    } else {
        if ((e = KL(HDG_PROF_SMOOTH_FIRST64, 1,
                    launch_smooth_first_t<double>(h, v, x, w_src, w_src ? &h->ws->rb->hnext : nullptr,
                                                  const_cast<double *>(v), cheb ? h->cheb_omega[0] : 0.0))) !=
            cudaSuccess)
            return e;
        double *prev = nullptr;
        for (int i = 1; i < h->prm.n_pre; ++i) {
            double *o = cheb ? (prev ? prev : x2) : x2;
            e = cheb ? KL(HDG_PROF_SMOOTH64, 1, launch_smooth_cheb_t<double>(h, v, x, o, h->cheb_omega[i],
                                                                             h->cheb_beta[i], prev))
                     : KL(HDG_PROF_SMOOTH64, 1, launch_smooth_t<double>(h, v, x, o));
            if (e != cudaSuccess) return e;
            if (cheb) {
                prev = x;
                x = o;
            } else {
                std::swap(x, x2);
            }
        }
        x2 = (x == k.t0) ? k.t1 : k.t0;
    }
    // residual, restriction to RT0, coarse Chebyshev steps, prolongation
    if ((e = KL(HDG_PROF_RESIDUAL64, 1, launch_residual_t<double>(h, v, x, k.res, true))) != cudaSuccess) return e;
    Rt0Dev &R = h->rt0;
    if ((e = KL(HDG_PROF_TRANSFER, 1, launch_rt0_restrict(h, k.res, R.rc))) != cudaSuccess) return e;
    double *cur = R.e0, *prev = nullptr, *spare[2] = {R.e1, R.e2};
    if ((e = KL(HDG_PROF_P1, 1, launch_rt0_cheb(h, R.rc, nullptr, nullptr, cur, h->cheb_c_omega[0], 0.0))) !=
        cudaSuccess)
        return e;
    for (int i = 1; i < h->prm.n_coarse; ++i) {
        double *o = prev ? prev : spare[0];
        if (o == cur) o = spare[1];
        if ((e = KL(HDG_PROF_P1, 1, launch_rt0_cheb(h, R.rc, cur, prev, o, h->cheb_c_omega[size_t(i)],
                                                      h->cheb_c_beta[size_t(i)]))) != cudaSuccess)
            return e;
        prev = cur;
        cur = o;
    }
    if ((e = KL(HDG_PROF_TRANSFER, 1, launch_rt0_prolong_add(h, cur, x))) != cudaSuccess) return e;
    // post-smoothing from x
    const int np = h->prm.n_post;
    if (np == 0) return cudaMemcpyAsync(z, x, sizeof(double) * NT, cudaMemcpyDeviceToDevice, s);
    if (!cheb) {
        for (int i = 0; i < np; ++i) {
            double *o = (i == np - 1) ? z : x2;
            if ((e = KL(HDG_PROF_SMOOTH64, 1, launch_smooth_t<double>(h, v, x, o))) != cudaSuccess) return e;
            if (i < np - 1) std::swap(x, x2);
        }
        return cudaSuccess;
    }
    // Chebyshev from x_0 = x: three vectors x, x2, k.res (free after the restriction)
    double *buf[3] = {x, x2, k.res};
    int cur_i = 0, prev_i = -1;
    for (int i = 0; i < np; ++i) {
        int out_i = 0;
        while (out_i == cur_i || out_i == prev_i) ++out_i;
        double *o = (i == np - 1) ? z : buf[out_i];
        if ((e = KL(HDG_PROF_SMOOTH64, 1, launch_smooth_cheb_t<double>(h, v, buf[cur_i], o, h->cheb_omega[size_t(i)],
                                                                         i ? h->cheb_beta[size_t(i)] : 0.0,
                                                                         i ? buf[prev_i] : nullptr))) != cudaSuccess)
            return e;
        prev_i = cur_i;
        cur_i = out_i;
    }
    return cudaSuccess;
}

// With w_src (Arnoldi steps j >= 1, n_pre >= 1), v is first formed as
// w_src / h_{j+1,j} by the first smoothing sweep, which stores it to v (with
// hsrc: w_src / hsrc[0] instead, the first step of a cycle).
template <typename T>
cudaError_t precond(hdg_handle *h, const T *v, T *z, const T *w_src = nullptr, const double *hsrc = nullptr) {
    if (h->prm.flux == 1) {
        if constexpr (std::is_same<T, double>::value) return precond_lf(h, v, z, w_src);
        return cudaErrorInvalidValue;
    }
    KSpace<T> &k = kspace<T>(h);
    cudaStream_t s = h->stream;
    const size_t NT = h->NT;
    T *x = k.t0, *x2 = k.t1;
    cudaError_t e;
    const bool cheb = h->prm.smoother == 1;
    // lines 1-2: pre-smoothing and residual
    if (cheb && h->prm.n_pre > 0) {
        // Chebyshev iteration from zero: x_1 = s_0 D^-1 v, then x_{k+1} = x_k +
        // 2 s_k D^-1 (v - S x_k) + delta^2 s_k s_{k-1} (x_k - x_{k-1})
        if ((e = KL(cat_first<T>(), 1,
                    launch_smooth_first_t<T>(h, v, x, w_src, w_src ? (hsrc ? hsrc : &h->ws->rb->hnext) : nullptr,
                                             const_cast<T *>(v), h->cheb_omega[0]))) != cudaSuccess)
            return e;
        T *prev = nullptr;
        for (int i = 1; i < h->prm.n_pre; ++i) {
            T *o = prev ? prev : x2;
            if ((e = KL(cat_smooth<T>(), 1, launch_smooth_cheb_t<T>(h, v, x, o, h->cheb_omega[i], h->cheb_beta[i],
                                                                     prev))) != cudaSuccess)
                return e;
            prev = x;
            x = o;
        }
        x2 = (x == k.t0) ? k.t1 : k.t0;
    } else if (h->prm.n_pre == 0) {
        if ((e = KL(HDG_PROF_KRYLOV, 1, launch_fill<T>(x, T(0), NT, s))) != cudaSuccess) return e;
    } else {
        if ((e = KL(cat_first<T>(), 1,
                    launch_smooth_first_t<T>(h, v, x, w_src, w_src ? (hsrc ? hsrc : &h->ws->rb->hnext) : nullptr,
                                             const_cast<T *>(v)))) != cudaSuccess)
            return e;
        for (int i = 1; i < h->prm.n_pre; ++i) {
            if ((e = KL(cat_smooth<T>(), 1, launch_smooth_t<T>(h, v, x, x2))) != cudaSuccess) return e;
            std::swap(x, x2);
        }
    }
    if ((e = KL(cat_res<T>(), 1, launch_residual_t<T>(h, v, x, k.res, true))) != cudaSuccess) return e;
    // line 3: restriction r_c = pi^T r (with the first P1 sweep when level 0 is above the tail)
    DevLevel &L0 = h->lev[0];
    const bool fuse0 = h->tail_start[sizeof(T) == 8 ? 0 : 1] > 0 && h->prm.p1_nu_pre >= 1;
    if ((e = KL(HDG_PROF_TRANSFER, 1, launch_restrict_t<T>(h, k.res, levB<T>(L0), fuse0 ? levD<T>(L0) : nullptr,
                                                           T(h->prm.p1_omega), fuse0 ? levX<T>(L0) : nullptr))) != cudaSuccess) return e;
    // line 4: coarse problem
    T *ec = nullptr;
    if ((e = p1_cycle<T>(h, &ec)) != cudaSuccess) return e;
    // lines 5-6: x += pi e_c and post-smoothing (the prolongation rides on the first sweep)
    const int np = h->prm.n_post;
    if (np == 0) {
        if ((e = KL(HDG_PROF_TRANSFER, 1, launch_prolong_add_t<T>(h, ec, x))) != cudaSuccess) return e;
        return dcopy(h, z, x, sizeof(T) * NT, cudaMemcpyDeviceToDevice);
    }
    bool learned = false, collect = false;
    if constexpr (std::is_same<T, float>::value) {
        learned = h->lc.on && !h->lc.suspended;
        collect = h->lc.collecting && h->lc.count < h->lc.cap;
    }
    if (cheb && !learned && !collect) {
        // Chebyshev iteration from x_0 = x + pi e_c: the first step rides on the
        // prolongation and keeps x_0 (in k.res, free after the restriction)
        T *cur = (np == 1) ? z : x2, *prev = (np == 1) ? nullptr : k.res;
        if ((e = KL(cat_smooth<T>(), 1, launch_smooth_prolong_t<T>(h, ec, v, x, cur, h->cheb_omega[0], prev))) !=
            cudaSuccess)
            return e;
        for (int i = 1; i < np; ++i) {
            T *o = (i == np - 1) ? z : prev;
            if ((e = KL(cat_smooth<T>(), 1, launch_smooth_cheb_t<T>(h, v, cur, o, h->cheb_omega[i], h->cheb_beta[i],
                                                                     prev))) != cudaSuccess)
                return e;
            prev = cur;
            cur = o;
        }
        return cudaSuccess;
    }
    if (!learned && !collect) {
        T *out = (np == 1) ? z : x2;
        if ((e = KL(cat_smooth<T>(), 1, launch_smooth_prolong_t<T>(h, ec, v, x, out))) != cudaSuccess) return e;
        std::swap(x, x2);
        for (int i = 1; i < np; ++i) {
            T *o = (i == np - 1) ? z : x2;
            if ((e = KL(cat_smooth<T>(), 1, launch_smooth_t<T>(h, v, x, o))) != cudaSuccess) return e;
            if (i < np - 1) std::swap(x, x2);
        }
        return cudaSuccess;
    }
    // n_post - 1 ordinary sweeps, then the residual r = v - S x before the last sweep
    T *cheb_prev = nullptr, *spare = k.res;   // Chebyshev: x_{n-2} for the last step; a free vector
    if (np == 1) {
        if ((e = KL(HDG_PROF_TRANSFER, 1, launch_prolong_add_t<T>(h, ec, x))) != cudaSuccess) return e;
    } else if (cheb) {
        // the first n_post - 1 steps of the Chebyshev iteration from x_0 = x + pi e_c,
        // rotating three vectors (x is free once x_0 is stored)
        T *cur = x2, *prev = k.res, *free_ = x;
        if ((e = KL(cat_smooth<T>(), 1, launch_smooth_prolong_t<T>(h, ec, v, x, cur, h->cheb_omega[0], prev))) !=
            cudaSuccess)
            return e;
        for (int i = 1; i < np - 1; ++i) {
            if ((e = KL(cat_smooth<T>(), 1, launch_smooth_cheb_t<T>(h, v, cur, free_, h->cheb_omega[i],
                                                                     h->cheb_beta[i], prev))) != cudaSuccess)
                return e;
            T *t = free_;
            free_ = prev;
            prev = cur;
            cur = t;
        }
        x = cur;
        cheb_prev = prev;
        spare = free_;
    } else {
        if ((e = KL(cat_smooth<T>(), 1, launch_smooth_prolong_t<T>(h, ec, v, x, x2))) != cudaSuccess) return e;
        std::swap(x, x2);
        for (int i = 1; i < np - 1; ++i) {
            if ((e = KL(cat_smooth<T>(), 1, launch_smooth_t<T>(h, v, x, x2))) != cudaSuccess) return e;
            std::swap(x, x2);
        }
    }
    if constexpr (std::is_same<T, float>::value) {
        if (learned) {
            // the learned sweep replaces the last smoothing step
            if ((e = KL(cat_res<T>(), 1, launch_residual_t<T>(h, v, x, spare, true))) != cudaSuccess) return e;
            return KL(HDG_PROF_KRYLOV, 1, h->lc.tc ? launch_learned_infer_tc(h, spare, x, z)
                                                   : launch_learned_infer(h, spare, x, z));
        }
        // collecting: store the residual (normalised), then the plain last step
        T *slot = h->lc.buf + size_t(h->lc.count) * NT;
        if ((e = KL(cat_res<T>(), 1, launch_residual_t<T>(h, v, x, slot, true))) != cudaSuccess) return e;
        Workspace &W = *h->ws;
        if ((e = dots<T>(h, slot, 1, slot, W.nrm2)) != cudaSuccess) return e;
        if ((e = launch_normalize32(slot, slot, W.nrm2, NT, s)) != cudaSuccess) return e;
        h->lc.count += 1;
    }
    if (cheb_prev)
        return KL(cat_smooth<T>(), 1, launch_smooth_cheb_t<T>(h, v, x, z, h->cheb_omega[size_t(np - 1)],
                                                              h->cheb_beta[size_t(np - 1)], cheb_prev));
    return KL(cat_smooth<T>(), 1, launch_smooth_t<T>(h, v, x, z));
}

// ---------------------------------------------------------------- Krylov helpers

template <typename T>
cudaError_t dots(hdg_handle *h, const T *V, int k, const T *w, double *out, HostValue *pub, int32_t seq,
                 double *root_a, double *root_b) {
    Workspace &W = *h->ws;
    if (k == 1)
        return KL(HDG_PROF_KRYLOV, 1, launch_dot1<T>(V, w, W.NT, W.partial, W.nchunk, W.counter, out, pub, seq, root_a,
                                                     root_b, h->stream));
    cudaError_t e = KL(HDG_PROF_KRYLOV, 1, launch_multidot<T>(V, W.NT, k, w, W.NT, W.partial, W.nchunk, h->stream));
    if (e != cudaSuccess) return e;
    return KL(HDG_PROF_KRYLOV, 1, launch_reduce_partials(W.partial, k, W.nchunk, out, h->stream, pub, seq, root_a,
                                                         root_b));
}

// Wait until the page-locked HostValue carries sequence number want: spin,
// checking the stream every 256 polls (an error, or a finished stream
// without the number, ends the wait with HDG_ECUDA).  There is no host-side
// time limit: the loop ends because the stream ends, and the stream ends
// because every wait inside the library's kernels is bounded by an iteration
// count (the coarse-cycle staging and the learned sweep's MMA waits set a
// status bit and return when theirs runs out).
int wait_host_value(hdg_handle *h, int32_t want) {
    Workspace &W = *h->ws;
    if (batch_recorder()) {
        const int rc = batch_yield(h, &W.host_val->seq, want);
        if (rc) return rc;
    }
    const volatile int32_t *seq = &W.host_val->seq;
    for (uint64_t it = 1;; ++it) {
        if (*seq == want) break;
        if ((it & 255) == 0) {
            const cudaError_t q = cudaStreamQuery(h->stream);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) return fail(h, HDG_ECUDA, std::string("norm: ") + cudaGetErrorString(q));
            if (*seq == want) break;
            return fail(h, HDG_ECUDA, "norm kernel finished without handing over its value");
        }
    }
    std::atomic_thread_fence(std::memory_order_acquire);
    return HDG_OK;
}

// ||v||: the reduction kernel hands the squared norm to the host through
// page-locked memory (no copy, no stream synchronisation)
// ||v|| from a squared norm that a kernel already launched hands over with
// sequence number want
int norm_wait(hdg_handle *h, int32_t want, double &out) {
    Workspace &W = *h->ws;
    if (h->prof.on) {
        TRY(cudaStreamSynchronize(h->stream));
        prof_flush(h);
    }
    int rc = wait_host_value(h, want);
    if (rc) return rc;
    out = std::sqrt(W.host_val->v);
    return HDG_OK;
}

template <typename T>
int norm_host(hdg_handle *h, const T *v, double &out) {
    Workspace &W = *h->ws;
    // the previous hand-over was seen, so no write to the word is in flight;
    // one fixed number keeps the launch arguments the same from call to call
    W.host_val->seq = 0;
    const int32_t want = 1;
    TRY(dots<T>(h, v, 1, v, W.nrm2, W.host_val_dev, want));
    return norm_wait(h, want, out);
}

// One Arnoldi step j of FGMRES: z_j = V(v_j), w = S z_j, classical
// Gram-Schmidt twice against v_0..v_j, h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j},
// Givens rotation j and the residual estimate copied to pinned host memory.
// Every argument is a fixed device address, so the step can be captured once
// in a CUDA graph and replayed.
template <typename T>
cudaError_t arnoldi_step(hdg_handle *h, int j, const T *src0 = nullptr) {
    Workspace &W = *h->ws;
    KSpace<T> &k = kspace<T>(h);
    cudaStream_t s = h->stream;
    const size_t NT = W.NT;
    const int ldh = W.m + 1;
    const size_t ld = W.ld;
    T *vj = k.V + size_t(j) * ld, *zj = k.Z + size_t(j) * ld;
    cudaError_t e;
    bool fuse_scale = h->prm.n_pre >= 1;
    if (std::is_same<T, double>::value && mode_pre32(h->prm)) {
        // FP64 FGMRES, FP32 preconditioner: v_j = w / h_{j,j-1} formed in FP64 and
        // rounded to FP32 in one pass, z_j widened back to FP64
        KSpace<float> &k32 = h->ws->k32;
        const double *wsrc = reinterpret_cast<const double *>(j > 0 ? k.w : vj);
        if ((e = KL(HDG_PROF_KRYLOV, 1, launch_scale_round(wsrc, j > 0 ? &W.rb->hnext : nullptr,
                                                            reinterpret_cast<double *>(vj), k32.b, NT, s))) !=
            cudaSuccess)
            return e;
        if ((e = precond<float>(h, k32.b, k32.x)) != cudaSuccess) return e;
        if ((e = KL(HDG_PROF_KRYLOV, 1, launch_widen(k32.x, reinterpret_cast<double *>(zj), NT, s))) != cudaSuccess)
            return e;
        fuse_scale = true;
    } else {
        // v_j = w / h_{j,j-1} rides on the first smoothing sweep (w and h from step j-1);
        // with src0, v_0 = src0 / ||src0|| (the scale the cycle left in W.scal)
        if (j == 0 && src0) e = precond<T>(h, vj, zj, src0, W.scal);
        else e = precond<T>(h, vj, zj, (fuse_scale && j > 0) ? k.w : nullptr);
        if (e != cudaSuccess) return e;
    }
    // w = S z_j with the first Gram-Schmidt pass h1 = V^T w in the same kernel
    if ((e = KL(cat_apply<T>(), 1, launch_apply_dots_t<T>(h, zj, k.w, k.V, ld, j + 1, W.partial, W.counter, W.h1))) !=
        cudaSuccess)
        return e;
    const bool reorth = h->prm.reorth != 0;
    if ((e = KL(HDG_PROF_KRYLOV, 1 + (reorth ? 1 : 0) + (fuse_scale ? 0 : 1),
                launch_gs_step<T>(k.V, ld, j, k.w, W.partial, W.counter, W.nblk_gs, W.h1, W.h2, W.nrm2, W.Hm, ldh,
                                  W.cs, W.sn, W.sv, W.bnorm, W.rb, W.host_rb_dev + j, k.V + size_t(j + 1) * ld, reorth,
                                  !fuse_scale, s))) != cudaSuccess)
        return e;
    (void)NT;
    return cudaSuccess;
}

// Wait for Arnoldi step j's readback: spin on the step number that the
// Gram-Schmidt kernel writes last into slot j of the page-locked copies,
// checking the stream every 256 polls (an error, or a finished stream without
// the number, ends the wait with HDG_ECUDA).  Like wait_host_value, it relies
// on every device-side wait of the library being bounded.
int wait_readback(hdg_handle *h, int j) {
    Workspace &W = *h->ws;
    if (batch_recorder()) {
        const int rc = batch_yield(h, &W.host_rb[j].seq, j + 1);
        if (rc) return rc;
    }
    const volatile int32_t *seq = &W.host_rb[j].seq;
    for (uint64_t it = 1;; ++it) {
        if (*seq == j + 1) break;
        if ((it & 255) == 0) {
            const cudaError_t q = cudaStreamQuery(h->stream);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) return fail(h, HDG_ECUDA, std::string("Arnoldi step: ") + cudaGetErrorString(q));
            if (*seq == j + 1) break;
            return fail(h, HDG_ECUDA, "Arnoldi step finished without its readback");
        }
    }
    std::atomic_thread_fence(std::memory_order_acquire);
    W.rb_pending[j] = 0;
    return HDG_OK;
}

// Run Arnoldi step j: directly while kernel timing is on, otherwise through
// its CUDA graph (captured on first use).
template <typename T>
int run_arnoldi_step(hdg_handle *h, int j, const T *src0 = nullptr) {
    Workspace &W = *h->ws;
    cudaStream_t s = h->stream;
    if (h->prof.on || !W.use_graphs || h->lc.collecting || batch_recorder()) {
        TRY(arnoldi_step<T>(h, j, src0));
        return HDG_OK;
    }
    const int gi = sizeof(T) == 8 ? 0 : ((h->lc.on && !h->lc.suspended) ? 2 : 1);
    Workspace::StepGraph &G = W.graphs[gi][(j == 0 && src0) ? W.m : j];
    if (G.exec && G.src != static_cast<const void *>(src0)) {   // captured for another right-hand side
        cudaGraphExecDestroy(G.exec);
        G.exec = nullptr;
    }
    if (!G.exec) {
        int64_t before[HDG_PROF_N];
        std::memcpy(before, h->prof.launches, sizeof(before));
        G.src = src0;
        TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = arnoldi_step<T>(h, j, src0);
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(s, &graph);
        for (int c = 0; c < HDG_PROF_N; ++c) {
            G.counts[c] = h->prof.launches[c] - before[c];
            h->prof.launches[c] = before[c];
        }
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return fail(h, HDG_ECUDA, std::string("capturing an Arnoldi step: ") +
                                          cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        cudaError_t e3 = cudaGraphInstantiate(&G.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e3 != cudaSuccess) {
            G.exec = nullptr;
            return fail(h, HDG_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e3));
        }
    }
    TRY(cudaGraphLaunch(G.exec, s));
    for (int c = 0; c < HDG_PROF_N; ++c) h->prof.launches[c] += G.counts[c];
    return HDG_OK;
}

// Launch Arnoldi step j after clearing its readback slot.  A step launched
// ahead whose number the host never waited for (its cycle ended first) may
// still write the slot: that write comes first in the stream, so it is waited
// for before the slot is cleared.
template <typename T>
int launch_arnoldi_step(hdg_handle *h, int j, const T *src0 = nullptr) {
    Workspace &W = *h->ws;
    if (W.rb_pending[j]) {
        const int rc = wait_readback(h, j);
        if (rc) return rc;
    }
    W.host_rb[j].seq = 0;
    W.rb_pending[j] = 1;
    return run_arnoldi_step<T>(h, j, src0);
}

// Steps launched ahead: HDG_SPECULATE unset, a margin (> 1) or 0 (off), read
// once.  fgmres_cycle launches step j + 1 before step j's readback arrives
// when the last two estimates, extrapolated geometrically, put step j's
// estimate above margin x the target (default margin 8).
double speculation_margin() {
    static const double v = [] {
        const char *e = std::getenv("HDG_SPECULATE");
        if (!e || !*e) return 8.0;
        const double m = std::atof(e);
        return m > 1.0 ? m : 0.0;
    }();
    return v;
}

// The mixed refinement's iterate as seen by an inner solve: the last cycle of
// the inner solve adds its correction scale * (x + Z y) straight into the
// float pairs (ff_finish) instead of updating x; done says it has.
struct PairsOut {
    float2 *x2 = nullptr;
    const double *scale = nullptr;
    bool first = false;    // the refinement iterate is still zero
    bool x_zero = false;   // (per cycle) the inner iterate x is still zero
    bool done = false;
};

// One FGMRES cycle (at most m iterations, possibly fewer) on S x = b starting
// from x, with the current residual r0 = b - S x of norm beta already in
// k.V[0] (scaled).  Stops when the estimate drops below tol_abs / bnorm.
// Returns the number of iterations; x is updated.
template <typename T>
int fgmres_cycle(hdg_handle *h, T *x, double beta, double bnorm, double rel_target, int max_it, int &its_done,
                 double &est_out, int &flag_out, bool beta_on_device = false, PairsOut *po = nullptr,
                 const T *src0 = nullptr) {
    Workspace &W = *h->ws;
    KSpace<T> &k = kspace<T>(h);
    cudaStream_t s = h->stream;
    const size_t NT = W.NT;
    const int m = W.m, ldh = m + 1;
    its_done = 0;
    flag_out = 0;
    est_out = beta / bnorm;
    // s = [beta, 0, ...]
    TRY(dzero(h, W.sv, sizeof(double) * (m + 1)));
    TRY(dzero(h, W.Hm, sizeof(double) * (m + 1) * m));
    if (beta_on_device) {
        // s_0 = ||b|| as the norm kernel left it in W.bnorm (first cycle, zero guess)
        TRY(dcopy(h, W.sv, W.bnorm, sizeof(double), cudaMemcpyDeviceToDevice));
    } else {
        W.host_buf[3] = beta;
        TRY(dcopy(h, W.sv, W.host_buf + 3, sizeof(double), cudaMemcpyHostToDevice));
    }
    int j = 0;
    double hist[72];
    // steps launched ahead (replayed step graphs only): step j + 1 is queued
    // behind step j before j's estimate reaches the host, so that the GPU does
    // not idle while the host reads it and launches the next step.  If step j
    // then meets the target, step j + 1 has run for nothing; its results (the
    // Hessenberg column j + 1, rotation j + 1, basis vectors past j) are not used.
    const double margin = speculation_margin();
    const bool ahead_ok = margin > 0.0 && !h->prof.on && W.use_graphs && !h->lc.on && !h->lc.collecting &&
                          !batch_recorder();
    bool launched[72] = {};
    const double est0 = est_out;
    for (; j < m && j < max_it; ++j) {
        int rc;
        if (!launched[j] && (rc = launch_arnoldi_step<T>(h, j, j == 0 ? src0 : nullptr))) return rc;
        if (ahead_ok && j >= 1 && j + 1 < m && j + 1 < max_it) {
            const double e1 = hist[j - 1], e2 = j >= 2 ? hist[j - 2] : est0;
            if (e2 > 0.0 && e1 * (e1 / e2) > margin * rel_target) {
                if ((rc = launch_arnoldi_step<T>(h, j + 1))) return rc;
                launched[j + 1] = true;
            }
        }
        if (h->prof.on) {
            TRY(cudaStreamSynchronize(s));
            prof_flush(h);
        } else if ((rc = wait_readback(h, j))) {
            return rc;
        }
        est_out = W.host_rb[j].est;
        flag_out = W.host_rb[j].flags;
        hist[j] = est_out;
        // learned sweep as preconditioner: if the residual estimate stalls (less
        // than 10 % decrease over three iterations), fall back to the plain
        // V-cycle for the rest of this solve (FGMRES restarts from the iterate)
        if (std::is_same<T, float>::value && h->lc.on && !h->lc.suspended && j >= 3 && est_out > rel_target &&
            est_out > 0.9 * hist[j - 3]) {
            h->lc.suspended = true;
            h->lc.fallback = true;
            ++j;
            break;
        }
        if (est_out <= rel_target || (flag_out & 6)) { ++j; break; }
    }
    its_done = j;
    if (j > 0 && !(flag_out & 4)) {
        // the inner solve ends with this cycle (the caller trusts the estimate)
        const bool last = est_out <= rel_target || j >= max_it;
        if constexpr (std::is_same<T, float>::value) {
            if (po && po->x2 && last) {
                TRY(KL(HDG_PROF_KRYLOV, 1, launch_ff_finish(W.Hm, ldh, W.sv, j, k.Z, W.ld, po->x_zero ? nullptr : x,
                                                           po->x2, po->scale, NT, po->first, s)));
                po->done = true;
                return HDG_OK;
            }
        }
        TRY(KL(HDG_PROF_KRYLOV, 1, launch_hessenberg_solve(W.Hm, ldh, W.sv, j, W.y, s)));
        TRY(KL(HDG_PROF_KRYLOV, 1, launch_multi_axpy<T>(x, k.Z, W.ld, j, W.y, 1.0, NT, s)));
    }
    return HDG_OK;
}

// Full FGMRES(m) on S x = b in precision T; stops on the true residual (FP64
// mode) or on the Arnoldi estimate (inner FP32 solves).  x must hold the
// initial guess; with x_zero (x = 0 on entry) the first residual is b itself
// and its norm is ||b||, so neither is recomputed.  unit_rhs (with x_zero):
// b = r / ||r|| by construction, finite with norm 1 up to rounding; its
// exact norm goes from the reduction kernel straight into the device scalars
// that use it (the estimate's denominator, the first basis vector's scale and
// s_0), and the host keeps the nominal 1 for its bookkeeping, so the solve
// starts without waiting for the GPU.  norm_ready: the kernel that formed b
// has already written that norm there.
template <typename T>
int fgmres(hdg_handle *h, const T *b, T *x, double rtol, int max_it, bool true_residual, bool x_zero,
           hdg_solve_info &info, bool unit_rhs = false, bool norm_ready = false, bool norm_pending = false,
           PairsOut *po = nullptr) {
    Workspace &W = *h->ws;
    KSpace<T> &k = kspace<T>(h);
    cudaStream_t s = h->stream;
    double bnorm = 1.0;
    int rc = HDG_OK;
    unit_rhs = unit_rhs && x_zero;
    info.iters = 0;
    info.outer = 0;
    info.est_rel_res = 0;
    info.true_rel_res = 0;
    if (unit_rhs) {
        // (norm_ready: the kernel that formed b already left ||b|| in W.bnorm and W.scal)
        if (!norm_ready) TRY(dots<T>(h, b, 1, b, W.nrm2, nullptr, 0, W.bnorm, W.scal));
    } else {
        // (norm_pending: the kernel that formed b hands ||b||^2 over with sequence number 1)
        rc = norm_pending ? norm_wait(h, 1, bnorm) : norm_host<T>(h, b, bnorm);
        if (rc) return rc;
        if (!std::isfinite(bnorm)) return fail(h, HDG_ENAN, "NaN or Inf in the right-hand side");
        if (bnorm == 0.0) {
            TRY(KL(HDG_PROF_KRYLOV, 1, launch_fill<T>(x, T(0), W.NT, s)));
            return HDG_OK;
        }
        // host_buf[4] is written again only after the next norm, whose hand-over
        // follows this copy in the stream
        W.host_buf[4] = bnorm;
        TRY(dcopy(h, W.bnorm, W.host_buf + 4, sizeof(double), cudaMemcpyHostToDevice));
    }
    int total = 0;
    for (bool first = true;; first = false) {
        // r = b - S x into V[0] (r = b for a zero initial guess)
        const T *r0 = k.V;
        double beta = bnorm;
        if (first && x_zero) {
            r0 = b;
        } else {
            TRY(KL(cat_res<T>(), 1, launch_residual_t<T>(h, b, x, k.V, false)));
            rc = norm_host<T>(h, k.V, beta);
            if (rc) return rc;
        }
        const double rel = beta / bnorm;
        info.true_rel_res = rel;
        if (!std::isfinite(rel)) return fail(h, HDG_ENAN, "NaN or Inf in the Krylov iteration");
        if (rel <= rtol) return HDG_OK;
        if (total >= max_it) return fail(h, HDG_ENOCONV, "maximum number of iterations reached");
        const bool beta_dev = first && unit_rhs;     // W.scal and W.bnorm already hold ||b||
        if (!beta_dev) {
            W.host_buf[1] = beta;
            TRY(dcopy(h, W.scal, W.host_buf + 1, sizeof(double), cudaMemcpyHostToDevice));
        }
        // v_0 = r0 / beta: formed by the first step's first smoothing sweep when r0 is
        // the right-hand side itself (a first cycle from a zero guess), else copied here
        const bool v0_fused = first && x_zero && h->prm.n_pre >= 1 && h->prm.flux == 0 &&
                              !(std::is_same<T, double>::value && mode_pre32(h->prm));
        if (!v0_fused) TRY(KL(HDG_PROF_KRYLOV, 1, launch_scale_copy<T>(r0, k.V, W.scal, W.NT, s)));
        int done, flag;
        double est;
        if (po) po->x_zero = first && x_zero;
        rc = fgmres_cycle<T>(h, x, beta, bnorm, rtol, max_it - total, done, est, flag, beta_dev,
                             true_residual ? nullptr : po, v0_fused ? r0 : nullptr);
        if (rc) return rc;
        total += done;
        info.iters = total;
        info.outer += 1;
        info.est_rel_res = est;
        if (flag & 4) return fail(h, HDG_ENAN, "NaN or Inf in the Krylov iteration");
        if (!true_residual && (est <= rtol || total >= max_it)) {
            // inner solve: trust the estimate
            info.true_rel_res = est;
            return HDG_OK;
        }
        if ((flag & 2) && est > rtol) {
            // breakdown without convergence: check the true residual once more
            TRY(KL(cat_res<T>(), 1, launch_residual_t<T>(h, b, x, k.V, false)));
            double beta2;
            rc = norm_host<T>(h, k.V, beta2);
            if (rc) return rc;
            info.true_rel_res = beta2 / bnorm;
            if (beta2 / bnorm <= rtol) return HDG_OK;
            return fail(h, HDG_EBREAKDOWN, "Krylov breakdown without convergence");
        }
    }
}

// FP64 iterative refinement with FP32 inner FGMRES solves.  The iterate is
// kept as float pairs in W.x2 (the form the refinement residual reads), so the
// correction x += d / sc runs in two-float arithmetic on the FP32 pipe;
// `updated` tells whether a correction has been added yet.  Each inner solve
// is S d = fp32(r sc) from a zero guess, sc a power of two, written with
// ||r sc|| by the kernel that forms r: the right-hand-side gather for r = g
// (norm_pending; sc = 1, g being in the FP32 range the two-float steps
// require) and the two-float residual afterwards (sc = 2^-ilogb(||g||), so
// that r sc stays near the relative residual).  Without norm_pending the
// first right-hand side is rounded by a separate pass as fp32(r / ||r||).
int solve_mixed_steps(hdg_handle *h, const double *g, hdg_solve_info &info, bool norm_pending, bool &updated) {
    Workspace &W = *h->ws;
    KSpace<float> &k = W.k32;
    cudaStream_t s = h->stream;
    double bnorm;
    int rc = norm_pending ? norm_wait(h, 1, bnorm) : norm_host<double>(h, g, bnorm);
    if (rc) return rc;
    info = hdg_solve_info{};
    if (!std::isfinite(bnorm)) return fail(h, HDG_ENAN, "NaN or Inf in the right-hand side");
    if (bnorm == 0.0) return HDG_OK;
    const double sc_res = std::ldexp(1.0, -std::ilogb(bnorm));
    int total = 0;
    for (int outer = 0;; ++outer) {
        double beta = bnorm, sc = 1.0;
        bool rhs32 = norm_pending;   // the FP32 start of the inner solve is written
        if (outer > 0) {
            // r = g - S x in two-float arithmetic from the pairs kept by the update
            // below, with the inner solve's start and ||r||^2 (handed to the host as
            // norm_host does) in the same pass
            sc = sc_res;
            rhs32 = true;
            F32Copy c32;
            c32.b32 = k.b;
            c32.z32 = k.x;
            c32.scale = sc;
            c32.root_a = W.bnorm;
            c32.root_b = W.scal;
            W.host_val->seq = 0;
            TRY(KL(HDG_PROF_RESIDUAL64, 1, launch_residual_ff(h, g, W.x2, nullptr, W.partial, W.counter, W.nrm2,
                                                              W.host_val_dev, 1, c32)));
            rc = norm_wait(h, 1, beta);
            if (rc) return rc;
        }
        info.true_rel_res = beta / bnorm;
        info.outer = outer;
        if (!std::isfinite(beta)) return fail(h, HDG_ENAN, "NaN or Inf in the refinement");
        if (beta / bnorm <= h->prm.rtol) return HDG_OK;
        if (total >= h->prm.max_iter || outer >= 100)
            return fail(h, HDG_ENOCONV, "maximum number of iterations reached");
        // the correction's scale: x += d / sc, or x += ||r|| d for b32 = r / ||r||
        W.host_buf[2] = rhs32 ? 1.0 / sc : beta;
        TRY(dcopy(h, W.beta, W.host_buf + 2, sizeof(double), cudaMemcpyHostToDevice));
        if (!rhs32) {
            // b32 = r / ||r||, the zero initial guess and ||b32|| (into W.bnorm and W.scal) in one pass
            TRY(KL(HDG_PROF_KRYLOV, 1, launch_d2f_norm(g, k.b, k.x, W.beta, W.NT, W.partial, W.nchunk, W.counter,
                                                       W.nrm2, W.bnorm, W.scal, s)));
        }
        hdg_solve_info inner{};
        const double inner_tol = std::max(h->prm.inner_rtol, 0.5 * h->prm.rtol * bnorm / beta);
        // (the inner solve's last cycle adds x += scale * d itself)
        PairsOut po;
        po.x2 = W.x2;
        po.scale = W.beta;
        po.first = !updated;
        rc = fgmres<float>(h, k.b, k.x, inner_tol, h->prm.max_iter - total, false, true, inner, true, true, false,
                           &po);
        if (rc && rc != HDG_ENOCONV) return rc;
        total += inner.iters;
        info.iters = total;
        info.est_rel_res = inner.est_rel_res;
        // x += scale * d (the first correction is x itself)
        if (!po.done) TRY(KL(HDG_PROF_KRYLOV, 1, launch_ff_axpy(W.x2, k.x, W.beta, W.NT, !updated, s)));
        updated = true;
    }
}

// the refinement above; on return the iterate is joined into x and lam (FP64,
// lam may be null), zero if no correction was added
int solve_mixed(hdg_handle *h, const double *g, double *x, hdg_solve_info &info, bool norm_pending, double *lam) {
    Workspace &W = *h->ws;
    bool updated = false;
    const int rc = solve_mixed_steps(h, g, info, norm_pending, updated);
    if (rc == HDG_ECUDA) return rc;
    if (updated) {
        TRY(KL(HDG_PROF_KRYLOV, 1, launch_ff_join(W.x2, x, lam, W.NT, h->stream)));
    } else {
        TRY(KL(HDG_PROF_KRYLOV, 1, launch_fill<double>(x, 0.0, W.NT, h->stream)));
        if (lam) TRY(KL(HDG_PROF_KRYLOV, 1, launch_fill<double>(lam, 0.0, W.NT, h->stream)));
    }
    return rc;
}

int ensure_staging(hdg_handle *h) {
    Workspace &W = *h->ws;
    if (W.ru) return HDG_OK;
    TRY(dalloc(&W.ru, size_t(h->N) * 2 * h->np));
    TRY(dalloc(&W.rh, size_t(h->N) * h->np));
    TRY(dalloc(&W.lam_ext, size_t(h->NT)));
    TRY(dalloc(&W.u, size_t(h->N) * 2 * h->np));
    TRY(dalloc(&W.hh, size_t(h->N) * h->np));
    return HDG_OK;
}

void free_handle(hdg_handle *h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    prof_flush(h);
    for (cudaEvent_t e : h->prof.pool) cudaEventDestroy(e);
    h->prof.pool.clear();
    imex_release(h);
    dfree(h->rt0.nbr); dfree(h->rt0.rev); dfree(h->rt0.ptr); dfree(h->rt0.code); dfree(h->rt0.piw);
    dfree(h->rt0.loc); dfree(h->rt0.fK); dfree(h->rt0.Sc); dfree(h->rt0.dinv);
    dfree(h->rt0.rc); dfree(h->rt0.e0); dfree(h->rt0.e1); dfree(h->rt0.e2);
    dfree(h->gal.ptr0);
    dfree(h->gal.code0);
    for (auto *p_ : h->gal.ptr) cudaFree(p_);
    for (auto *p_ : h->gal.idx) cudaFree(p_);
    for (auto *p_ : h->gal.w) cudaFree(p_);
    if (h->prof.evict_buf) cudaFree(h->prof.evict_buf);
    if (h->prof.evict_sink) cudaFree(h->prof.evict_sink);
    dfree(h->d_ref); dfree(h->d_X); dfree(h->d_fcell); dfree(h->d_facet_of); dfree(h->d_flip);
    dfree(h->d_facet_cell); dfree(h->d_facet_edge); dfree(h->d_facet_verts); dfree(h->d_v2f_ptr); dfree(h->d_v2f);
    dfree(h->d_nbr); dfree(h->d_Xb); dfree(h->d_Rm); dfree(h->d_W); dfree(h->d_Scell); dfree(h->d_Sval);
    dfree(h->d_Xb2); dfree(h->d_Rm2); dfree(h->d_W2); dfree(h->d_Sval2);
    dfree(h->d_cgeo); dfree(h->d_ctab_v); dfree(h->d_ctab_b);
    dfree(h->d_Dinv); dfree(h->d_Sval32); dfree(h->d_Dinv32); dfree(h->d_Sval16); dfree(h->d_status); dfree(h->d_coarse_inv);
    dfree(h->tail_img[0].d); dfree(h->tail_img[1].d);
    dfree(h->d_coarse_work);
    dfree(h->d_coarse_fac);
    for (auto &L : h->lev) {
        dfree(L.col); dfree(L.diag); dfree(L.elem); dfree(L.fK); dfree(L.contrib_ptr); dfree(L.contrib); dfree(L.A); dfree(L.dinv);
        dfree(L.A32); dfree(L.dinv32); dfree(L.parent); dfree(L.child_ptr); dfree(L.child_idx); dfree(L.child_w); dfree(L.child_w32);
        dfree(L.pf_ptr); dfree(L.pf_n0); dfree(L.pf_ids); dfree(L.pf0_base); dfree(L.plcol);
        dfree(L.pc_ptr); dfree(L.pc_ids); dfree(L.pcc_ptr); dfree(L.pcc_slot); dfree(L.pcc_w); dfree(L.pcc_w32);
        dfree(L.pg_ptr); dfree(L.pg_nown); dfree(L.pg_ids); dfree(L.pg0_base); dfree(L.pglcol);
        dfree(L.pfcol); dfree(L.pgcol); dfree(L.pgpar); dfree(L.pgrow_par);
        dfree(L.x); dfree(L.x2); dfree(L.b); dfree(L.r); dfree(L.x32); dfree(L.x232); dfree(L.b32); dfree(L.r32);
    }
    if (h->ws) {
        Workspace &W = *h->ws;
        dfree(W.g); dfree(W.x); dfree(W.r); dfree(W.ycell); dfree(W.x2); dfree(W.z2);
        dfree(W.k64.V); dfree(W.k64.Z); dfree(W.k64.w); dfree(W.k64.t0); dfree(W.k64.t1); dfree(W.k64.res);
        dfree(W.k32.V); dfree(W.k32.Z); dfree(W.k32.w); dfree(W.k32.t0); dfree(W.k32.t1); dfree(W.k32.res);
        dfree(W.k32.b); dfree(W.k32.x);
        dfree(W.Hm); dfree(W.cs); dfree(W.sn); dfree(W.sv); dfree(W.h1); dfree(W.h2); dfree(W.nrm2);
        dfree(W.est); dfree(W.counter); dfree(W.rb);
        if (W.host_rb) cudaFreeHost(W.host_rb);
        if (W.host_val) cudaFreeHost(W.host_val);
        dfree(W.scal); dfree(W.bnorm);
        for (auto &gv : W.graphs)
            for (auto &G : gv)
                if (G.exec) cudaGraphExecDestroy(G.exec); dfree(W.beta); dfree(W.y); dfree(W.partial); dfree(W.flags);
        dfree(W.ru); dfree(W.rh); dfree(W.lam_ext); dfree(W.u); dfree(W.hh); dfree(W.lam_int);
        dfree(W.ru_x); dfree(W.rh_x);
        if (W.host_buf) cudaFreeHost(W.host_buf);
        if (W.host_flags) cudaFreeHost(W.host_flags);
        delete h->ws;
    }
    {
        Learned &L = h->lc;
        dfree(L.theta); dfree(L.m); dfree(L.v); dfree(L.grad); dfree(L.act); dfree(L.gfac); dfree(L.rev);
        dfree(L.wimg); dfree(L.gpart);
        dfree(L.buf); dfree(L.c); dfree(L.rn); dfree(L.gc); dfree(L.tmp); dfree(L.coef); dfree(L.nrm);
    }
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

void drop_graphs(hdg_handle *h);

// The tail image of precision pi (0: FP64, 1: FP32) for the current tail
// start: header table, every level's staged arrays and, when it fits, the
// coarsest FP64 inverse, copied device to device into one buffer.  Needs the
// assembled level operators (hdg_condense).
int build_tail_image(hdg_handle *h, int pi) {
    if (pi == 1 && !h->lev[0].A32) return HDG_OK;          // no FP32 levels on this handle
    const size_t tsz = pi == 0 ? sizeof(double) : sizeof(float);
    const int ts = h->tail_start[pi], n = int(h->lev.size()) - ts;
    TailLayout lay;
    if (!tail_layout(tail_sizes(h->lev, ts), tsz, size_t(h->lev.back().nv), lay))
        return fail(h, HDG_EINVAL, "coarsest P1 levels too large for the single-CTA coarse cycle");
    const std::vector<TailHdr> &hdr = lay.hdr;
    const size_t img_bytes = lay.img_bytes;
    const int32_t inv_off = lay.inv_off;
    const size_t off = lay.smem_bytes;
    auto source = [&](const TailPiece &q) -> const void * {
        const DevLevel &L = h->lev[size_t(ts + q.level)];
        switch (q.kind) {
        case kTailA: return pi == 0 ? static_cast<const void *>(L.A) : static_cast<const void *>(L.A32);
        case kTailD: return pi == 0 ? static_cast<const void *>(L.dinv) : static_cast<const void *>(L.dinv32);
        case kTailCol: return L.col;
        case kTailCw: return pi == 0 ? static_cast<const void *>(L.child_w) : static_cast<const void *>(L.child_w32);
        case kTailCp: return L.child_ptr;
        case kTailCi: return L.child_idx;
        case kTailPar: return L.parent;
        default: return h->d_coarse_inv;
        }
    };
    TailImage &im = h->tail_img[pi];
    if (im.cap < img_bytes) {
        dfree(im.d);
        im.cap = 0;
        TRY(dalloc(&im.d, img_bytes));
        im.cap = img_bytes;
        if (h->ws) drop_graphs(h);                         // captured launches hold the old address
    }
    cudaStream_t s = h->stream;
    TRY(cudaMemcpyAsync(im.d, hdr.data(), sizeof(TailHdr) * n, cudaMemcpyHostToDevice, s));
    for (const TailPiece &q : lay.pieces) {
        if (q.kind == kTailCol) continue;                  // packed together with the values
        if (q.kind == kTailA) {
            const DevLevel &L = h->lev[size_t(ts + q.level)];
            TRY(launch_tail_pack(L.col, source(q), tsz, L.nv, L.width, im.d + hdr[size_t(q.level)].ocol, im.d + q.off, s));
            continue;
        }
        TRY(cudaMemcpyAsync(im.d + q.off, source(q), q.bytes, cudaMemcpyDeviceToDevice, s));
    }
    TRY(cudaStreamSynchronize(s));                         // hdr is host memory on this stack
    if (im.ts != ts || im.img_bytes != img_bytes) {
        if (h->ws) drop_graphs(h);
    }
    im.ts = ts;
    im.img_bytes = uint32_t(img_bytes);
    im.smem_bytes = uint32_t(off);
    im.inv_off = inv_off;
    im.ob0 = hdr[0].ob;
    im.ox0 = hdr[0].ox;
    return HDG_OK;
}

// First level of the single-CTA coarse cycle, per precision: the largest
// suffix of P1 levels whose levels have at most tail_max vertices and whose
// operators, transfers and vectors fit in one CTA's shared memory.
int set_tail_start(hdg_handle *h, int tail_max64, int tail_max32) {
    const int nlev = int(h->lev.size());
    for (int pi = 0; pi < 2; ++pi) {
        const size_t tsz = pi == 0 ? sizeof(double) : sizeof(float);
        const int tail_max = pi == 0 ? tail_max64 : tail_max32;
        int ts = nlev - 1;
        while (ts > 0 && h->lev[ts - 1].nv <= tail_max && nlev - (ts - 1) <= kTailMaxLevels &&
               tail_smem_bytes(h->lev, ts - 1, tsz) <= size_t(220) * 1024)
            --ts;
        if (tail_smem_bytes(h->lev, ts, tsz) > kTailSmemMax)
            return fail(h, HDG_EINVAL, "coarsest P1 level too large for the single-CTA coarse cycle");
        h->tail_start[pi] = ts;
        if (h->condensed) {
            int rc = build_tail_image(h, pi);
            if (rc) return rc;
        }
    }
    return HDG_OK;
}

void drop_graphs(hdg_handle *h) {
    for (auto &gv : h->ws->graphs)
        for (auto &G : gv)
            if (G.exec) {
                cudaGraphExecDestroy(G.exec);
                G.exec = nullptr;
            }
}

// The tables of C_K formed from geometry in the solves' step 1 (two-float
// handles): per cell and edge the pairs of H t_y, -H t_x and tau_s |e| (t the
// edge vector, as the condensation's C_K uses them), and per row (edge i, trace
// node j) the cell nodes b with a nonzero reference facet entry N_ibj and its
// pair.  Those are the p + 1 nodes on the edge; another pattern leaves cz_ok
// false and the solves read the stored W_K instead.
float2 host_split(double v) {
    const float hi = static_cast<float>(v);
    return float2{hi, static_cast<float>(v - static_cast<double>(hi))};
}
int build_cz(hdg_handle *h, const RefElem &re) {
    cudaStream_t s = h->stream;
    const int np = h->np, pp = h->pp, N = h->N;
    const HostMesh &hm = h->hm;
    double nmax = 0.0;
    for (double v : re.N) nmax = std::max(nmax, std::fabs(v));
    std::vector<int32_t> tb(size_t(3) * pp * pp, 0);
    std::vector<float2> tv(size_t(3) * pp * pp, float2{0.0f, 0.0f});
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < pp; ++j) {
            int c = 0;
            for (int b = 0; b < np; ++b) {
                const double v = re.N[(size_t(i) * np + b) * pp + j];
                if (!(std::fabs(v) > 1e-13 * nmax)) continue;
                if (c == pp) return HDG_OK;
                tb[(size_t(i) * pp + j) * pp + c] = b;
                tv[(size_t(i) * pp + j) * pp + c] = host_split(v);
                ++c;
            }
        }
    const double H = h->prm.H, ts = h->tau_s;
    std::vector<float2> cg(size_t(N) * 9);
    for (int K = 0; K < N; ++K) {
        const double *x = hm.X.data() + size_t(K) * 6;
        for (int i = 0; i < 3; ++i) {
            const int v1 = (i + 1) % 3, v2 = (i + 2) % 3;
            const double tx = x[2 * v2] - x[2 * v1], ty = x[2 * v2 + 1] - x[2 * v1 + 1];
            float2 *o = cg.data() + (size_t(K) * 3 + i) * 3;
            o[0] = host_split(H * ty);
            o[1] = host_split(-H * tx);
            o[2] = host_split(ts * std::sqrt(tx * tx + ty * ty));
        }
    }
    TRY(upload(&h->d_ctab_b, tb, s));
    TRY(upload(&h->d_ctab_v, tv, s));
    TRY(upload(&h->d_cgeo, cg, s));
    TRY(cudaStreamSynchronize(s));      // the host vectors go out of scope
    h->cz_ok = true;
    return HDG_OK;
}

int setup_device(hdg_handle *h, const hdg_params *prm) {
    cudaStream_t s = h->stream;
    const HostMesh &hm = h->hm;
    RefElem re = build_ref_elem(h->p);
    TRY(upload(&h->d_ref, re.packed(), s));
    TRY(upload(&h->d_X, hm.X, s));
    std::vector<double> fcell(size_t(h->N) * 3, 0.0);
    if (prm->f_vertex)
        for (int K = 0; K < h->N; ++K)
            for (int i = 0; i < 3; ++i) {
                fcell[size_t(K) * 3 + i] = prm->f_vertex[hm.cells[3 * K + i]];
                if (fcell[size_t(K) * 3 + i] != 0.0) h->has_f = true;
            }
    TRY(upload(&h->d_fcell, fcell, s));
    TRY(upload(&h->d_facet_of, hm.facet_of, s));
    TRY(upload(&h->d_flip, hm.flip, s));
    TRY(upload(&h->d_facet_cell, hm.facet_cell, s));
    TRY(upload(&h->d_facet_edge, hm.facet_edge, s));
    TRY(upload(&h->d_facet_verts, hm.facet_verts, s));
    TRY(upload(&h->d_v2f_ptr, hm.v2f_ptr, s));
    TRY(upload(&h->d_v2f, hm.v2f, s));
    const size_t N = h->N, NF = h->NF, nK = h->nK, m = h->m, pp = h->pp;
    TRY(dalloc(&h->d_nbr, 4 * NF));
    TRY(dalloc(&h->d_Xb, nK * m * N));
    TRY(dalloc(&h->d_Rm, nK * nK * N));
    TRY(dalloc(&h->d_W, m * nK * N));
    TRY(dalloc(&h->d_Scell, N * m * m));
    auto packed = [&](size_t n, size_t G) { return (n + G - 1) / G * G * NF; };
    TRY(dalloc(&h->d_Sval, packed(5 * pp * pp, 2)));
    TRY(dalloc(&h->d_Dinv, packed(pp * pp, 2)));
    TRY(dalloc(&h->d_status, 1));
    const bool mixed = prm->precision != HDG_FP64;
    if (mixed) {
        TRY(dalloc(&h->d_Sval32, packed(5 * pp * pp, 4)));
        TRY(dalloc(&h->d_Dinv32, packed(pp * pp, 4)));
        if (mode_ff(*prm)) {
            // pairs of row entries (odd rows padded by one zero entry), tiles of 32 cells
            const size_t Nt = (N + 31) / 32 * 32;
            TRY(dalloc(&h->d_Xb2, nK * ((m + 1) / 2 * 2) * Nt));
            TRY(dalloc(&h->d_Rm2, nK * ((nK + 1) / 2 * 2) * Nt));
            TRY(dalloc(&h->d_W2, m * ((nK + 1) / 2 * 2) * Nt));
            TRY(dalloc(&h->d_Sval2, packed(5 * pp * pp, 2)));
            if (prm->flux == 0) {
                const int rc = build_cz(h, re);
                if (rc) return rc;
            }
        }
        if (prm->precision == HDG_MIXED_BF16) TRY(dalloc(&h->d_Sval16, packed(5 * pp * pp, 8)));
    }
    // Coriolis parameter per cell (mean of its vertices) on every P1 level; on a
    // coarser level a vertex takes the value of the finer-level vertex that
    // coincides with it (parent pair (a, a))
    std::vector<std::vector<double>> lev_fK(hm.levels.size());
    {
        std::vector<double> fv(size_t(h->nv), 0.0);
        if (prm->f_vertex) fv.assign(prm->f_vertex, prm->f_vertex + h->nv);
        for (size_t l = 0; l < hm.levels.size(); ++l) {
            const HostLevel &hl = hm.levels[l];
            if (l > 0) {
                std::vector<double> fc(size_t(hl.nv), 0.0);
                for (size_t i = 0; i + 1 < hl.parent.size(); i += 2)
                    if (hl.parent[i] == hl.parent[i + 1]) fc[hl.parent[i]] = fv[i / 2];
                fv.swap(fc);
            }
            lev_fK[l].resize(size_t(hl.nc));
            for (int K = 0; K < hl.nc; ++K)
                lev_fK[l][K] = (fv[hl.cells[3 * K]] + fv[hl.cells[3 * K + 1]] + fv[hl.cells[3 * K + 2]]) / 3.0;
        }
    }
    h->lev.resize(hm.levels.size());
    for (size_t l = 0; l < hm.levels.size(); ++l) {
        const HostLevel &hl = hm.levels[l];
        DevLevel &L = h->lev[l];
        L.nv = hl.nv;
        L.width = hl.width;
        L.nnz = int(hl.col.size());
        if (L.nnz == 0 || int(hl.diag.size()) != L.nv) return fail(h, HDG_EINVAL, "empty P1 level operator");
        for (int v = 0; v < L.nv; ++v)
            if (hl.diag[v] < 0) return fail(h, HDG_EINVAL, "P1 vertex without a cell");
        TRY(upload(&L.col, hl.col, s));
        TRY(upload(&L.diag, hl.diag, s));
        TRY(upload(&L.elem, hl.elem, s));
        TRY(upload(&L.contrib_ptr, hl.contrib_ptr, s));
        TRY(upload(&L.contrib, hl.contrib, s));
        TRY(upload(&L.fK, lev_fK[l], s));
        TRY(dalloc(&L.A, size_t(L.nnz)));
        TRY(dalloc(&L.dinv, size_t(L.nv)));
        if (l > 0) {
            TRY(upload(&L.parent, hl.parent, s));
            TRY(upload(&L.child_ptr, hl.child_ptr, s));
            TRY(upload(&L.child_idx, hl.child_idx, s));
            TRY(upload(&L.child_w, hl.child_w, s));
            std::vector<float> w32(hl.child_w.begin(), hl.child_w.end());
            TRY(upload(&L.child_w32, w32, s));
            L.nci = int(hl.child_idx.size());
        }
        if (hl.patch.nb > 0) {
            const HostPatches &P = hl.patch;
            L.nb = P.nb; L.max_f1 = P.max_f1; L.max_f0 = P.max_f0; L.max_g1 = P.max_g1;
            TRY(upload(&L.pf_ptr, P.f_ptr, s)); TRY(upload(&L.pf_n0, P.f_n0, s)); TRY(upload(&L.pf_ids, P.f_ids, s));
            TRY(upload(&L.pf0_base, P.f0_base, s)); TRY(upload(&L.plcol, P.lcol, s));
            TRY(upload(&L.pc_ptr, P.c_ptr, s)); TRY(upload(&L.pc_ids, P.c_ids, s));
            TRY(upload(&L.pcc_ptr, P.cc_ptr, s)); TRY(upload(&L.pcc_slot, P.cc_slot, s));
            TRY(upload(&L.pcc_w, P.cc_w, s));
            std::vector<float> cw32(P.cc_w.begin(), P.cc_w.end());
            TRY(upload(&L.pcc_w32, cw32, s));
            TRY(upload(&L.pg_ptr, P.g_ptr, s)); TRY(upload(&L.pg_nown, P.g_nown, s)); TRY(upload(&L.pg_ids, P.g_ids, s));
            TRY(upload(&L.pg0_base, P.g0_base, s)); TRY(upload(&L.pglcol, P.glcol, s));
            TRY(upload(&L.pfcol, P.fcol, s)); TRY(upload(&L.pgcol, P.gcol, s));
            TRY(upload(&L.pgpar, P.gpar, s)); TRY(upload(&L.pgrow_par, P.grow_par, s));
        }
        TRY(dalloc(&L.x, size_t(L.nv)));
        TRY(dalloc(&L.x2, size_t(L.nv)));
        TRY(dalloc(&L.b, size_t(L.nv)));
        TRY(dalloc(&L.r, size_t(L.nv)));
        if (mixed) {
            TRY(dalloc(&L.A32, size_t(L.nnz)));
            TRY(dalloc(&L.dinv32, size_t(L.nv)));
            TRY(dalloc(&L.x32, size_t(L.nv)));
            TRY(dalloc(&L.x232, size_t(L.nv)));
            TRY(dalloc(&L.b32, size_t(L.nv)));
            TRY(dalloc(&L.r32, size_t(L.nv)));
        }
    }
    {
        // largest level of the single-CTA coarse cycle per precision (FP64 levels:
        // 256, FP32 levels: 1,024, as measured fastest); HDG_TAIL_MAX_VERTICES sets both
        int tail_max64 = kTailMaxVertices64, tail_max32 = kTailMaxVertices;
        if (const char *ev = std::getenv("HDG_TAIL_MAX_VERTICES"))
            tail_max64 = tail_max32 = std::max(16, std::min(4096, std::atoi(ev)));
        // HDG_P1_FUSED=0 selects the unfused P1 kernels (same arithmetic; for timing comparisons)
        if (const char *ev = std::getenv("HDG_P1_FUSED")) h->p1_fused = std::atoi(ev) != 0;
        // HDG_FACET_BLOCK = 64 / 128 / 256: threads per block of the facet-row kernels
        // (one of the autotuner's candidates; same arithmetic)
        if (const char *ev = std::getenv("HDG_FACET_BLOCK")) {
            const int bs = std::atoi(ev);
            if (bs == 64 || bs == 128 || bs == 256) h->bs_facet = bs;
        }
        int rc = set_tail_start(h, tail_max64, tail_max32);
        if (rc) return rc;
    }
    if (prm->flux == 1) {
        Rt0Host rh;
        const std::string re_ = build_rt0(hm, h->p, rh);
        if (!re_.empty()) return fail(h, HDG_EINVAL, re_);
        for (int K = 0; K < h->N; ++K)
            rh.fK[size_t(K)] = (fcell[size_t(K) * 3] + fcell[size_t(K) * 3 + 1] + fcell[size_t(K) * 3 + 2]) / 3.0;
        Rt0Dev &R = h->rt0;
        TRY(upload(&R.nbr, rh.nbr, s)); TRY(upload(&R.rev, rh.rev, s));
        TRY(upload(&R.ptr, rh.ptr, s)); TRY(upload(&R.code, rh.code, s));
        TRY(upload(&R.piw, rh.piw, s)); TRY(upload(&R.loc, rh.loc, s)); TRY(upload(&R.fK, rh.fK, s));
        TRY(dalloc(&R.Sc, 5 * NF)); TRY(dalloc(&R.dinv, NF));
        TRY(dalloc(&R.rc, NF)); TRY(dalloc(&R.e0, NF)); TRY(dalloc(&R.e1, NF)); TRY(dalloc(&R.e2, NF));
        TRY(cudaStreamSynchronize(s));      // the host vectors go out of scope
    }
    if (prm->coarse_mode == 2) {
        GalerkinHost gh;
        const std::string ge = build_galerkin_lists(hm, gh);
        if (!ge.empty()) return fail(h, HDG_EINVAL, ge);
        TRY(upload(&h->gal.ptr0, gh.ptr0, s));
        TRY(upload(&h->gal.code0, gh.code0, s));
        for (size_t l = 0; l < gh.ptr.size(); ++l) {
            int32_t *pp_ = nullptr, *ii = nullptr;
            double *ww = nullptr;
            TRY(upload(&pp_, gh.ptr[l], s));
            h->gal.ptr.push_back(pp_);
            TRY(upload(&ii, gh.idx[l], s));
            h->gal.idx.push_back(ii);
            TRY(upload(&ww, gh.w[l], s));
            h->gal.w.push_back(ww);
        }
        TRY(cudaStreamSynchronize(s));      // the host vectors go out of scope
    }
    const size_t nc = h->lev.back().nv;
    TRY(dalloc(&h->d_coarse_inv, nc * nc));
    TRY(dalloc(&h->d_coarse_work, nc * nc));
    TRY(dalloc(&h->d_coarse_fac, nc));

    h->ws = new Workspace();
    Workspace &W = *h->ws;
    W.m = prm->restart;
    W.NT = h->NT;
    W.nchunk = int(std::min<size_t>(std::max<size_t>((W.NT + 4095) / 4096, 1), 608));
    TRY(dalloc(&W.g, W.NT));
    TRY(dalloc(&W.x, W.NT));
    TRY(dalloc(&W.r, W.NT));
    TRY(dalloc(&W.lam_int, W.NT));
    TRY(dalloc(&W.ycell, N * m));
    if (mode_ff(h->prm)) TRY(dalloc(&W.x2, W.NT));
    if (h->cz_ok && h->prm.keep_rhs) TRY(dalloc(&W.z2, size_t(h->nK) * N));
    const size_t mm = W.m;
    W.ld = (W.NT + 3) / 4 * 4;
    // one 16-byte group of w per thread (enough loads in flight for the few-vector
    // steps at the start of a cycle), at most 8 blocks of 256 per SM of a GB300
    W.nblk_gs = int(std::min<size_t>(std::max<size_t>((W.ld / 4 + 255) / 256, 1), kMaxGsBlocks));
    if (mode_krylov64(h->prm)) {
        TRY(dalloc(&W.k64.V, (mm + 1) * W.ld));
        TRY(dalloc(&W.k64.Z, mm * W.ld));
        TRY(dalloc(&W.k64.w, W.ld));
        TRY(cudaMemsetAsync(W.k64.V, 0, sizeof(double) * (mm + 1) * W.ld, s));
        TRY(cudaMemsetAsync(W.k64.w, 0, sizeof(double) * W.ld, s));
        if (mode_pre32(h->prm)) {
            // the FP32 preconditioner's work vectors, its input and its output
            TRY(dalloc(&W.k32.t0, W.NT));
            TRY(dalloc(&W.k32.t1, W.NT));
            TRY(dalloc(&W.k32.res, W.NT));
            TRY(dalloc(&W.k32.b, W.NT));
            TRY(dalloc(&W.k32.x, W.NT));
        }
    } else {
        // FP64 vectors still needed by the FP64 operator entry points
        TRY(dalloc(&W.k64.V, W.ld));
        TRY(dalloc(&W.k64.w, W.ld));
        TRY(dalloc(&W.k32.V, (mm + 1) * W.ld));
        TRY(dalloc(&W.k32.Z, mm * W.ld));
        TRY(dalloc(&W.k32.w, W.ld));
        TRY(cudaMemsetAsync(W.k32.V, 0, sizeof(float) * (mm + 1) * W.ld, s));
        TRY(cudaMemsetAsync(W.k32.w, 0, sizeof(float) * W.ld, s));
        TRY(dalloc(&W.k32.t0, W.NT));
        TRY(dalloc(&W.k32.t1, W.NT));
        TRY(dalloc(&W.k32.res, W.NT));
        TRY(dalloc(&W.k32.b, W.NT));
        TRY(dalloc(&W.k32.x, W.NT));
    }
    TRY(dalloc(&W.k64.t0, W.NT));
    TRY(dalloc(&W.k64.t1, W.NT));
    TRY(dalloc(&W.k64.res, W.NT));
    TRY(dalloc(&W.Hm, (mm + 1) * mm));
    TRY(dalloc(&W.cs, mm + 1));
    TRY(dalloc(&W.sn, mm + 1));
    TRY(dalloc(&W.sv, mm + 1));
    TRY(dalloc(&W.h1, mm + 1));
    TRY(dalloc(&W.h2, mm + 1));
    TRY(dalloc(&W.nrm2, 1));
    TRY(dalloc(&W.est, 1));
    TRY(dalloc(&W.scal, 1));
    TRY(dalloc(&W.bnorm, 1));
    for (auto &gv : W.graphs) gv.resize(W.m + 1);
    {
        const char *ev = std::getenv("HDG_DISABLE_GRAPHS");
        W.use_graphs = !(ev && ev[0] == '1');
    }
    TRY(dalloc(&W.beta, 1));
    TRY(dalloc(&W.y, mm + 1));
    // partial sums: (m + 1) vectors x the largest grid of the multi-dot (nchunk) or
    // of the Gram-Schmidt kernels (nblk_gs, or up to 1216 blocks after autotuning)
    TRY(dalloc(&W.partial, (mm + 1) * size_t(std::max({W.nchunk, W.nblk_gs, kMaxGsBlocks, int((h->NF + 255) / 256),
                                                        int((h->NF + kResFFFacets - 1) / kResFFFacets)}))));
    TRY(dalloc(&W.counter, 1));
    TRY(cudaMemsetAsync(W.counter, 0, sizeof(unsigned int), s));
    TRY(dalloc(&W.rb, 1));
    TRY(cudaMallocHost(reinterpret_cast<void **>(&W.host_rb), sizeof(ReadBack) * mm));
    std::memset(W.host_rb, 0, sizeof(ReadBack) * mm);
    W.rb_pending.assign(mm, 0);
    TRY(cudaHostGetDevicePointer(reinterpret_cast<void **>(&W.host_rb_dev), W.host_rb, 0));
    TRY(cudaMallocHost(reinterpret_cast<void **>(&W.host_val), sizeof(HostValue)));
    std::memset(W.host_val, 0, sizeof(HostValue));
    TRY(cudaHostGetDevicePointer(reinterpret_cast<void **>(&W.host_val_dev), W.host_val, 0));
    TRY(dalloc(&W.flags, 1));
    TRY(cudaMallocHost(reinterpret_cast<void **>(&W.host_buf), 8 * sizeof(double)));
    TRY(cudaHostGetDevicePointer(reinterpret_cast<void **>(&W.host_buf_dev), W.host_buf, 0));
    TRY(cudaMallocHost(reinterpret_cast<void **>(&W.host_flags), 4 * sizeof(int32_t)));
    TRY(cudaStreamSynchronize(s));
    return HDG_OK;
}

int check_status(hdg_handle *h) {
    int32_t st = 0;
    TRY(cudaMemcpyAsync(&st, h->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    TRY(cudaStreamSynchronize(h->stream));
    prof_flush(h);
    if (st & 1) return fail(h, HDG_ESINGULAR, "zero pivot in a cell matrix A_K");
    if (st & 2) return fail(h, HDG_ESINGULAR, "singular facet block of the trace operator");
    if (st & 4) return fail(h, HDG_ESINGULAR, "singular coarsest P1 operator");
    return HDG_OK;
}

// Ritz values of k Arnoldi steps (classical Gram-Schmidt twice, FP64) on the
// operator apply(x, y, tmp) of n entries, from the host start vector v0 (in
// device order), normalised here.  Stops early at an invariant subspace.
int arnoldi_ritz_dev(hdg_handle *h, const std::vector<double> &v0_in, int k,
                     const std::function<cudaError_t(const double *, double *, double *)> &apply,
                     std::vector<std::complex<double>> &ritz, const char *what) {
    Workspace &W = *h->ws;
    cudaStream_t s = h->stream;
    const size_t n = v0_in.size(), ld = (n + 3) / 4 * 4;
    std::vector<double> v0(v0_in);
    double nrm = 0.0;
    for (double x : v0) nrm += x * x;
    nrm = std::sqrt(nrm);
    for (double &x : v0) x /= nrm;
    double *V = nullptr, *tmp = nullptr, *w = nullptr, *part = nullptr, *dh = nullptr;
    cudaError_t e = dalloc(&V, size_t(k + 1) * ld);
    if (e == cudaSuccess) e = dalloc(&tmp, ld);
    if (e == cudaSuccess) e = dalloc(&w, ld);
    if (e == cudaSuccess) e = dalloc(&part, size_t(k + 2) * size_t(W.nchunk));
    if (e == cudaSuccess) e = dalloc(&dh, size_t(k + 2));
    if (e == cudaSuccess) e = cudaMemsetAsync(V, 0, sizeof(double) * size_t(k + 1) * ld, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(w, 0, sizeof(double) * ld, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(V, v0.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s);
    std::vector<double> Hm(size_t(k + 1) * k, 0.0), hc(size_t(k + 2));
    int m = k;
    for (int j = 0; j < k && e == cudaSuccess; ++j) {
        e = apply(V + size_t(j) * ld, w, tmp);
        for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
            e = launch_multidot<double>(V, ld, j + 1, w, n, part, W.nchunk, s);
            if (e == cudaSuccess) e = launch_reduce_partials(part, j + 1, W.nchunk, dh, s);
            if (e == cudaSuccess) e = launch_multi_axpy<double>(w, V, ld, j + 1, dh, -1.0, n, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(hc.data(), dh, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            for (int i = 0; i <= j; ++i) Hm[size_t(i) * k + j] += hc[size_t(i)];
        }
        // ||w|| into dh[k + 1] (the square root written by the reduction)
        if (e == cudaSuccess) e = launch_multidot<double>(w, ld, 1, w, n, part, W.nchunk, s);
        if (e == cudaSuccess) e = launch_reduce_partials(part, 1, W.nchunk, dh, s, nullptr, 0, dh + k + 1);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hc.data(), dh + k + 1, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) break;
        double colmax = 0.0;
        for (int i = 0; i <= j; ++i) colmax = std::max(colmax, std::fabs(Hm[size_t(i) * k + j]));
        if (!(hc[0] > 1e-14 * colmax)) {
            m = j + 1;                     // invariant subspace: the Ritz values are exact
            break;
        }
        if (j + 1 < k) Hm[size_t(j + 1) * k + j] = hc[0];
        e = launch_scale_copy<double>(w, V + size_t(j + 1) * ld, dh + k + 1, n, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dfree(V); dfree(tmp); dfree(w); dfree(part); dfree(dh);
    if (e != cudaSuccess) return fail(h, HDG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    std::vector<double> Hs(size_t(m) * m);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) Hs[size_t(i) * m + j] = Hm[size_t(i) * k + j];
    for (double x : Hs)
        if (!std::isfinite(x)) return fail(h, HDG_ENAN, std::string(what) + ": non-finite Arnoldi entry");
    ritz = hessenberg_eigenvalues(Hs, m);
    return HDG_OK;
}

// Step coefficients of n Chebyshev steps on the ellipse (theta, delta2):
// s_0 = 1/theta, s_k = 1 / (2 theta - delta^2 s_{k-1}), omega_0 = s_0,
// omega_k = 2 s_k, beta_k = delta^2 s_k s_{k-1}.
void chebyshev_coefficients(double theta, double delta2, int n, std::vector<double> &omega, std::vector<double> &beta) {
    omega.assign(size_t(n), 0.0);
    beta.assign(size_t(n), 0.0);
    double sp = 1.0 / theta;
    omega[0] = sp;
    for (int i = 1; i < n; ++i) {
        const double si = 1.0 / (2.0 * theta - delta2 * sp);
        omega[size_t(i)] = 2.0 * si;
        beta[size_t(i)] = delta2 * si * sp;
        sp = si;
    }
}

// The Chebyshev start vector v_i = 1 + ((37 i) mod 101) / 101 for index i.
inline double cheb_start(size_t i) { return 1.0 + double((37 * i) % 101) / 101.0; }

// The Chebyshev smoother's ellipse: Ritz values of cheb_steps Arnoldi steps on
// D^-1 S (i = facet * pp + node in the lambda layout), then the fit of
// spectrum.cpp; or the ellipse given in the parameters.
int chebyshev_setup(hdg_handle *h) {
    h->cheb_ritz.clear();
    if (h->prm.cheb_theta > 0) {
        h->cheb_theta = h->prm.cheb_theta;
        h->cheb_delta2 = h->prm.cheb_delta2;
    } else {
        const size_t NF = h->NF, pp = h->pp;
        std::vector<double> v0(h->NT);
        for (size_t e_ = 0; e_ < NF; ++e_)
            for (size_t r = 0; r < pp; ++r) v0[r * NF + e_] = cheb_start(e_ * pp + r);
        int rc = arnoldi_ritz_dev(h, v0, h->prm.cheb_steps, [&](const double *x, double *y, double *tmp) {
            cudaError_t e = launch_apply_t<double>(h, x, tmp);
            return e == cudaSuccess ? launch_smooth_first_t<double>(h, tmp, y, nullptr, nullptr, nullptr, 1.0) : e;
        }, h->cheb_ritz, "Chebyshev estimate");
        if (rc) return rc;
        chebyshev_ellipse(h->cheb_ritz, 0.1, 1.1, h->cheb_theta, h->cheb_delta2);
        if (!(h->cheb_theta > 0)) return fail(h, HDG_EBREAKDOWN, "Chebyshev estimate: no eigenvalue with Re > 0");
    }
    chebyshev_coefficients(h->cheb_theta, h->cheb_delta2, std::max({h->prm.n_pre, h->prm.n_post, 1}), h->cheb_omega,
                           h->cheb_beta);
    return HDG_OK;
}

// The Lax-Friedrichs coarse solve: ellipse of D_c^-1 S_c from cheb_steps
// Arnoldi steps (start vector over the facets), n_coarse step coefficients.
int lf_coarse_setup(hdg_handle *h) {
    std::vector<double> v0(size_t(h->NF));
    for (size_t f = 0; f < v0.size(); ++f) v0[f] = cheb_start(f);
    int rc = arnoldi_ritz_dev(h, v0, h->prm.cheb_steps, [&](const double *x, double *y, double *) {
        return launch_rt0_apply_dinv(h, x, y);
    }, h->cheb_c_ritz, "RT0 coarse estimate");
    if (rc) return rc;
    chebyshev_ellipse(h->cheb_c_ritz, 0.1, 1.1, h->cheb_c_theta, h->cheb_c_delta2);
    if (!(h->cheb_c_theta > 0)) return fail(h, HDG_EBREAKDOWN, "RT0 coarse estimate: no eigenvalue with Re > 0");
    chebyshev_coefficients(h->cheb_c_theta, h->cheb_c_delta2, h->prm.n_coarse, h->cheb_c_omega, h->cheb_c_beta);
    return HDG_OK;
}

int require_condensed(hdg_handle *h) {
    if (!h) return HDG_EINVAL;
    if (!h->condensed) return fail(h, HDG_ESTATE, "hdg_condense has not run on this handle");
    return HDG_OK;
}

// copy_u / copy_h (mixed modes, optional): device buffers that receive r_u, r_h
// as the right-hand-side kernel reads them (used when those are host memory)
int solve_internal(hdg_handle *h, const double *r_u, const double *r_h, hdg_solve_info &info,
                   double *copy_u = nullptr, double *copy_h = nullptr) {
    Workspace &W = *h->ws;
    cudaStream_t s = h->stream;
    h->lc.suspended = false;
    h->lc.fallback = false;
    // the right-hand side g with ||g|| handed to the host by the same kernel
    // (upwind flux; the Lax-Friedrichs right-hand side has no such kernel)
    const bool norm_pending = h->prm.flux == 0;
    NormOut nrm;
    if (norm_pending) {
        W.host_val->seq = 0;   // the previous hand-over was seen
        nrm = NormOut{W.partial, W.counter, W.nrm2, W.host_val_dev, 1};
        if (mode_ff(h->prm)) {
            // and the first inner solve's start: fp32(g), the zero guess, ||g||
            nrm.f32.b32 = W.k32.b;
            nrm.f32.z32 = W.k32.x;
            nrm.f32.root_a = W.bnorm;
            nrm.f32.root_b = W.scal;
        }
    }
    W.have_z = false;
    if (!mode_ff(h->prm)) {
        TRY(KL(HDG_PROF_RHS, 2, launch_rhs(h, r_u, r_h, W.g, W.ycell, nrm)));
    } else if (W.z2) {
        // keeping z_K = R_M r_K for the recovery of this solve
        TRY(KL(HDG_PROF_RHS, 2, launch_rhs_z(h, r_u, r_h, W.g, W.ycell, W.z2, copy_u, copy_h, nrm)));
        W.have_z = true;
    } else {
        TRY(KL(HDG_PROF_RHS, 2, launch_rhs_ff(h, r_u, r_h, W.g, W.ycell, copy_u, copy_h, nrm)));
    }
    int rc;
    if (mode_krylov64(h->prm)) {
        TRY(KL(HDG_PROF_KRYLOV, 1, launch_fill<double>(W.x, 0.0, W.NT, s)));
        rc = fgmres<double>(h, W.g, W.x, h->prm.rtol, h->prm.max_iter, true, true, info, false, false, norm_pending);
    } else {
        rc = solve_mixed(h, W.g, W.x, info, norm_pending, W.lam_int);
    }
    if (!batch_recorder()) {   // a batched solve checks the status words after its last wave
        int32_t st = 0;
        TRY(cudaMemcpyAsync(&st, h->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        TRY(cudaStreamSynchronize(s));
        if (st & (8 | 16)) {
            rc = fail(h, HDG_ETIMEOUT, (st & 8) ? "a bounded device-side wait ran out (coarse-cycle staging)"
                                                : "a bounded device-side wait ran out (tensor-core MMA of the "
                                                  "learned sweep)");
            TRY(cudaMemsetAsync(h->d_status, 0, sizeof(int32_t), s));
        }
    }
    info.status = rc;
    info.fallback_used = h->lc.fallback ? 1 : 0;
    // (the mixed refinement has written lam_int with x)
    if (mode_krylov64(h->prm)) TRY(dcopy(h, W.lam_int, W.x, sizeof(double) * W.NT, cudaMemcpyDeviceToDevice));
    W.have_lambda = true;
    return rc;
}

// ---------------------------------------------------------------- merged batches
// Each problem of a merged batch runs the host logic of hdg_solve_dev
// unchanged, as a fiber (a user-level context on its own stack) of the one
// calling thread.  While a fiber runs, its launches are recorded; where the
// host logic would wait for a value from the GPU, the fiber hands control
// back to the batch loop.  Once every unfinished fiber of a group waits with
// launches recorded, the loop merges and launches them as the group's next
// wave.  A fiber is resumed as soon as the word it waits on arrives, while the
// rest of its wave may still run, so that its next launches are recorded by
// the time the wave ends.
constexpr size_t kFiberStack = size_t(512) << 10;

struct Fiber {
    ucontext_t ctx;
    std::unique_ptr<unsigned char[]> stack;
    hdg_handle *h = nullptr;
    const double *r_u = nullptr, *r_h = nullptr;
    double *lambda = nullptr;
    int32_t *status_dev = nullptr;   // device address of this problem's page-locked status word
    hdg_solve_info info{};
    int rc = HDG_OK;
    bool done = false;
    bool launched = false;           // the launches it recorded before its wait have been launched
    const volatile int32_t *wait_addr = nullptr;
    int32_t wait_want = 0;
    Recorder rec;
};

thread_local Fiber *t_fiber = nullptr;            // the fiber running on this thread
thread_local ucontext_t *t_sched = nullptr;       // the batch loop it returns to
thread_local const char *t_wave_error = nullptr;  // set once a wave has failed

int batch_yield(hdg_handle *h, const volatile int32_t *addr, int32_t want) {
    Fiber *f = t_fiber;
    if (!f || !t_sched) return fail(h, HDG_ESTATE, "launch recording outside a batched solve");
    f->wait_addr = addr;
    f->wait_want = want;
    f->launched = false;
    swapcontext(&f->ctx, t_sched);
    if (t_wave_error) return fail(h, HDG_ECUDA, std::string("batched solve: ") + t_wave_error);
    return HDG_OK;
}

// one problem: the steps of hdg_solve_dev, then its status word to the host
void fiber_entry() {
    Fiber *f = t_fiber;
    hdg_handle *h = f->h;
    f->rc = solve_internal(h, f->r_u, f->r_h, f->info);
    if (f->rc != HDG_ECUDA) {
        const cudaError_t e = KL(HDG_PROF_LAYOUT, 1, launch_to_external(h, h->ws->x, f->lambda));
        if (e != cudaSuccess) f->rc = fail(h, HDG_ECUDA, std::string("launch_to_external: ") + cudaGetErrorString(e));
        h->ws->have_rhs = false;
    }
    const cudaError_t e2 = launch_copy(f->status_dev, h->d_status, sizeof(int32_t), h->stream);
    if (e2 != cudaSuccess && f->rc == HDG_OK)
        f->rc = fail(h, HDG_ECUDA, std::string("status copy: ") + cudaGetErrorString(e2));
    f->done = true;
}

}  // namespace

struct hdg_batch {
    // Problems are dealt into groups; each group has its own stream, its own
    // waves and graphs, so that the host prepares one group's next wave while
    // the waves of the others run.
    struct Group {
        std::vector<int> idx;                     // its problems
        std::vector<Recorder *> recs;
        cudaStream_t stream = nullptr;
        cudaEvent_t ev = nullptr;                 // end of its last wave
        bool inflight = false;
        hdg::WaveRunner runner;
    };
    std::vector<hdg_handle *> hs;
    std::vector<std::unique_ptr<Fiber>> fibers;   // never moved: a context holds pointers into itself
    std::vector<std::unique_ptr<Group>> groups;
    std::vector<int> group_of;                    // per problem
    int device = 0;
    std::vector<cudaEvent_t> ev_in;               // one per handle: its stream's work before the batch
    int32_t *status_host = nullptr, *status_dev = nullptr;   // page-locked, one word per handle
    int64_t ns_fibers = 0, ns_launch = 0, ns_wait = 0;       // host time: running fibers, merging/launching, waiting
};

namespace {

void batch_release(hdg_batch *b) {
    if (!b) return;
    for (auto &g : b->groups) {
        g->runner.clear();
        if (g->ev) cudaEventDestroy(g->ev);
        if (g->stream) cudaStreamDestroy(g->stream);
    }
    for (cudaEvent_t e : b->ev_in)
        if (e) cudaEventDestroy(e);
    if (b->status_host) cudaFreeHost(b->status_host);
    delete b;
}

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

}  // namespace

// ====================================================================== ABI

extern "C" {


void hdg_default_params(hdg_params *prm) {
    if (!prm) return;
    std::memset(prm, 0, sizeof(*prm));
    prm->p = 1;
    prm->tau = 1.0;
    prm->g = 1.0;
    prm->H = 1.0;
    prm->tau_s = 0.0;
    prm->f_vertex = nullptr;
    prm->precision = HDG_FP64;
    prm->rtol = 1e-8;
    prm->restart = 30;
    prm->max_iter = 500;
    prm->n_pre = 2;
    prm->n_post = 2;
    prm->omega = 2.0 / 3.0;
    prm->p1_nu_pre = 2;
    prm->p1_nu_post = 2;
    prm->p1_omega = 2.0 / 3.0;
    prm->inner_rtol = 1e-4;
    prm->coarse_mode = 0;
    prm->reorth = 0;
    prm->smoother = 0;
    prm->cheb_theta = 0.0;
    prm->cheb_delta2 = 0.0;
    prm->cheb_steps = 20;
    prm->flux = 0;
    prm->n_coarse = 20;
    prm->keep_rhs = 1;
}

int hdg_setup(const hdg_mesh_desc *mesh, const hdg_params *prm, void *stream, hdg_handle **out) {
    if (!out) return fail(nullptr, HDG_EINVAL, "out is NULL");
    *out = nullptr;
    std::string e = check_params(prm);
    if (!e.empty()) return fail(nullptr, HDG_EINVAL, e);
    hdg_handle *h = new hdg_handle();
    h->prm = *prm;
    h->prm.f_vertex = nullptr;      // not kept: the values are copied
    e = build_host_mesh(mesh, h->hm);
    if (!e.empty()) {
        delete h;
        return fail(nullptr, HDG_EINVAL, e);
    }
    if (prm->flux == 1 && h->hm.dim != 2) {
        delete h;
        return fail(nullptr, HDG_EINVAL, "the Lax-Friedrichs solver handles flat (dim = 2) meshes");
    }
    h->p = prm->p;
    h->pp = (prm->flux == 1 ? 2 : 1) * (prm->p + 1);     // trace dofs per facet
    h->pf = h->pp - 1;
    h->np = n_cell_nodes(prm->p);
    h->nK = 3 * h->np;
    h->m = 3 * h->pp;
    h->N = h->hm.nc;
    h->NF = h->hm.nf;
    h->NT = h->NF * h->pp;
    h->nv = h->hm.nv;
    h->dim = h->hm.dim;
    h->tau_s = prm->tau_s > 0 ? prm->tau_s : std::sqrt(prm->g * prm->H);
    // FP64 facet-row kernels need ~240 registers per thread (one 256-thread block
    // per SM); blocks of 128 measured faster for them (smooth64 65 -> 53 us)
    h->bs_facet = prm->precision == HDG_FP64 ? 128 : 256;
    if (stream) {
        h->stream = static_cast<cudaStream_t>(stream);
    } else {
        cudaError_t ce = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (ce != cudaSuccess) {
            delete h;
            return fail(nullptr, HDG_ECUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(ce));
        }
        h->own_stream = true;
    }
    int rc = setup_device(h, prm);
    if (!rc) {
        // the device this handle lives on, and the no-allocation scratch array
        // loaded onto it now rather than inside a later call
        cudaError_t ce = cudaGetDevice(&h->device);
        if (ce == cudaSuccess) ce = noalloc_prepare(h);
        if (ce != cudaSuccess) rc = fail(h, HDG_ECUDA, std::string("no-allocation scratch: ") + cudaGetErrorString(ce));
    }
    if (rc) {
        std::string msg = h->err;
        free_handle(h);
        return fail(nullptr, rc == HDG_ECUDA && msg.find("memory") != std::string::npos ? HDG_ENOMEM : rc, msg);
    }
    *out = h;
    return HDG_OK;
}

int hdg_condense(hdg_handle *h) {
    if (!h) return HDG_EINVAL;
    cudaStream_t s = h->stream;
    h->condensed = false;
    if (h->ws) h->ws->have_z = false;      // z_K = R_M r_K belongs to the old operator
    TRY(cudaMemsetAsync(h->d_status, 0, sizeof(int32_t), s));
    if (h->prm.flux == 1) {
        // Lax-Friedrichs: cell operators and the facet-row operator on 2(p+1) blocks,
        // the RT0 coarse operator and its Chebyshev coarse solve
        TRY(KL(HDG_PROF_CONDENSE, 2, launch_condense_lf(h)));
        TRY(KL(HDG_PROF_CONDENSE, 2, launch_rt0_assemble(h)));
        int rc = check_status(h);
        if (rc) return rc;
        if ((rc = lf_coarse_setup(h)) != HDG_OK) return rc;
        if (h->prm.smoother == 1 && (rc = chebyshev_setup(h)) != HDG_OK) return rc;
        h->condensed = true;
        return HDG_OK;
    }
    TRY(KL(HDG_PROF_CONDENSE, 1, launch_condense(h)));
    TRY(KL(HDG_PROF_CONDENSE, 1, launch_assemble(h)));
    const double tau = h->prm.tau, gH = h->prm.g * h->prm.H;
    if (h->prm.coarse_mode == 2) {
        TRY(KL(HDG_PROF_CONDENSE, int(2 * h->lev.size()), launch_p1_galerkin(h)));
    } else {
        for (auto &L : h->lev)
            TRY(KL(HDG_PROF_CONDENSE, 2, launch_p1_assemble(h, L, tau, gH, h->prm.coarse_mode == 0 ? 1 : 0)));
    }
    const DevLevel &Lc = h->lev.back();
    TRY(KL(HDG_PROF_CONDENSE, Lc.nv <= 256 ? 2 : 2 + 2 * Lc.nv,
           launch_dense_inverse(h, Lc, h->d_coarse_work, h->d_coarse_inv, Lc.nv)));
    if (h->prm.precision != HDG_FP64) {
        TRY(KL(HDG_PROF_CONDENSE, h->d_Sval16 ? 3 : 2, launch_repack(h)));
        for (auto &L : h->lev) {
            TRY(KL(HDG_PROF_CONDENSE, 1, launch_to_f32(L.A, L.A32, size_t(L.nnz), s)));
            TRY(KL(HDG_PROF_CONDENSE, 1, launch_to_f32(L.dinv, L.dinv32, size_t(L.nv), s)));
        }
        if (mode_ff(h->prm)) {
            // (hi, lo) float pairs for the two-float FP64 steps
            const size_t N = h->N, nK = h->nK, m = h->m, pp = h->pp, NS = 5 * pp * pp;
            if (!condense_writes_pairs(h)) {
                TRY(KL(HDG_PROF_CONDENSE, 1, launch_split_pairs(h->d_Xb, h->d_Xb2, int(nK), int(m), N, s)));
                TRY(KL(HDG_PROF_CONDENSE, 1, launch_split_pairs(h->d_Rm, h->d_Rm2, int(nK), int(nK), N, s)));
                TRY(KL(HDG_PROF_CONDENSE, 1, launch_split_pairs(h->d_W, h->d_W2, int(m), int(nK), N, s)));
            }
            TRY(KL(HDG_PROF_CONDENSE, 1, launch_split(h->d_Sval, h->d_Sval2, (NS + 1) / 2 * 2 * size_t(h->NF), s)));
        }
    }
    for (int pi = 0; pi < 2; ++pi) {
        int rc = build_tail_image(h, pi);
        if (rc) return rc;
    }
    int rc = check_status(h);
    if (rc) return rc;
    if (h->prm.smoother == 1 && (rc = chebyshev_setup(h)) != HDG_OK) return rc;
    h->condensed = true;
    return HDG_OK;
}

int hdg_get_rt0_chebyshev(const hdg_handle *hc, double *ellipse, double *ritz, int32_t *n_ritz) {
    hdg_handle *h = const_cast<hdg_handle *>(hc);
    if (!h) return HDG_EINVAL;
    if (h->prm.flux != 1) return fail(h, HDG_ESTATE, "the handle does not use the Lax-Friedrichs solver");
    if (!h->condensed) return fail(h, HDG_ESTATE, "hdg_condense has not run on this handle");
    if (ellipse) {
        ellipse[0] = h->cheb_c_theta;
        ellipse[1] = h->cheb_c_delta2;
    }
    const int n = int(std::min<size_t>(h->cheb_c_ritz.size(), 64));
    if (ritz)
        for (int i = 0; i < n; ++i) {
            ritz[2 * i] = h->cheb_c_ritz[size_t(i)].real();
            ritz[2 * i + 1] = h->cheb_c_ritz[size_t(i)].imag();
        }
    if (n_ritz) *n_ritz = n;
    return HDG_OK;
}

int hdg_get_chebyshev(const hdg_handle *hc, double *ellipse, double *ritz, int32_t *n_ritz) {
    hdg_handle *h = const_cast<hdg_handle *>(hc);
    if (!h) return HDG_EINVAL;
    if (h->prm.smoother != 1) return fail(h, HDG_ESTATE, "the handle does not use the Chebyshev smoother");
    if (!h->condensed) return fail(h, HDG_ESTATE, "hdg_condense has not run on this handle");
    if (ellipse) {
        ellipse[0] = h->cheb_theta;
        ellipse[1] = h->cheb_delta2;
    }
    const int n = int(std::min<size_t>(h->cheb_ritz.size(), 64));
    if (ritz)
        for (int i = 0; i < n; ++i) {
            ritz[2 * i] = h->cheb_ritz[size_t(i)].real();
            ritz[2 * i + 1] = h->cheb_ritz[size_t(i)].imag();
        }
    if (n_ritz) *n_ritz = n;
    return HDG_OK;
}

int hdg_set_tau(hdg_handle *h, double tau) {
    if (!h) return HDG_EINVAL;
    if (!(tau > 0)) return fail(h, HDG_EINVAL, "tau must be positive");
    h->prm.tau = tau;
    return hdg_condense(h);
}

int hdg_solve_dev(hdg_handle *h, const double *r_u, const double *r_h, double *lambda, hdg_solve_info *info) {
    int rc = require_condensed(h);
    if (rc) return rc;
    if (!r_u || !r_h || !lambda) return fail(h, HDG_EINVAL, "NULL pointer argument");
    hdg_solve_info loc{};
    rc = solve_internal(h, r_u, r_h, loc);
    if (rc == HDG_ECUDA) {
        if (info) *info = loc;
        return rc;
    }
    TRY(KL(HDG_PROF_LAYOUT, 1, launch_to_external(h, h->ws->x, lambda)));
    h->ws->have_rhs = false;
    if (info) *info = loc;
    return rc;
}

namespace {
// hdg_solve, ending with a stream synchronisation when sync is set
int solve_host(hdg_handle *h, const double *r_u, const double *r_h, double *lambda, hdg_solve_info *info,
               bool sync) {
    int rc = require_condensed(h);
    if (rc) return rc;
    if (!r_u || !r_h || !lambda) return fail(h, HDG_EINVAL, "NULL pointer argument");
    rc = ensure_staging(h);
    if (rc) return rc;
    Workspace &W = *h->ws;
    cudaStream_t s = h->stream;
    hdg_solve_info loc{};
    // page-locked inputs of a mixed handle: the right-hand-side kernel reads them
    // in place (and keeps device copies for hdg_recover); otherwise staged copies
    const double *ru_a = host_alias(r_u), *rh_a = host_alias(r_h);
    if (mode_ff(h->prm) && ru_a && rh_a) {
        rc = solve_internal(h, ru_a, rh_a, loc, W.ru, W.rh);
    } else {
        TRY(cudaMemcpyAsync(W.ru, r_u, sizeof(double) * size_t(h->N) * 2 * h->np, cudaMemcpyHostToDevice, s));
        TRY(cudaMemcpyAsync(W.rh, r_h, sizeof(double) * size_t(h->N) * h->np, cudaMemcpyHostToDevice, s));
        rc = solve_internal(h, W.ru, W.rh, loc);
    }
    if (rc == HDG_ECUDA) {
        if (info) *info = loc;
        return rc;
    }
    if (double *lam_a = host_alias(lambda)) {
        TRY(KL(HDG_PROF_LAYOUT, 1, launch_to_external(h, W.x, lam_a)));
    } else {
        TRY(KL(HDG_PROF_LAYOUT, 1, launch_to_external(h, W.x, W.lam_ext)));
        TRY(cudaMemcpyAsync(lambda, W.lam_ext, sizeof(double) * W.NT, cudaMemcpyDeviceToHost, s));
    }
    if (sync) TRY(cudaStreamSynchronize(s));
    W.have_rhs = true;
    if (info) *info = loc;
    return rc;
}
}  // namespace

int hdg_solve(hdg_handle *h, const double *r_u, const double *r_h, double *lambda, hdg_solve_info *info) {
    return solve_host(h, r_u, r_h, lambda, info, true);
}

int hdg_solve_recover(hdg_handle *h, const double *r_u, const double *r_h, double *lambda, double *u, double *h_out,
                      hdg_solve_info *info) {
    if (h && (!u || !h_out)) return fail(h, HDG_EINVAL, "NULL output pointer");
    // steps 1 and 2 without the closing synchronisation, step 3 from what they left
    // in the handle (this solve's lambda and right-hand side); one synchronisation
    const int rc = solve_host(h, r_u, r_h, lambda, info, false);
    if (rc == HDG_ECUDA || rc == HDG_EINVAL || rc == HDG_ESTATE) return rc;
    const int rc2 = hdg_recover(h, nullptr, nullptr, nullptr, u, h_out);
    return rc ? rc : rc2;
}

int hdg_recover_dev(hdg_handle *h, const double *r_u, const double *r_h, const double *lambda, double *u,
                    double *h_out) {
    int rc = require_condensed(h);
    if (rc) return rc;
    if (!u || !h_out) return fail(h, HDG_EINVAL, "NULL output pointer");
    if (!r_u != !r_h) return fail(h, HDG_EINVAL, "r_u and r_h must both be given or both be NULL");
    Workspace &W = *h->ws;
    // r_u = r_h = NULL: the last solve's right-hand side, as z_K = R_M r_K kept by
    // its step 1, else as the copies hdg_solve keeps
    if (!r_u && !W.have_z && !W.have_rhs)
        return fail(h, HDG_ESTATE, "no right-hand side given and none kept from the last solve");
    const double *lam = W.lam_int;
    if (lambda) {
        TRY(KL(HDG_PROF_LAYOUT, 1, launch_to_internal(h, lambda, W.k64.res)));
        lam = W.k64.res;
    } else if (!W.have_lambda) {
        return fail(h, HDG_ESTATE, "no lambda given and no previous solve");
    }
    if (!r_u && W.have_z) {
        TRY(KL(HDG_PROF_RECOVER, 1, launch_recover_z(h, W.z2, lam, u, h_out)));
        return HDG_OK;
    }
    const double *ru = r_u ? r_u : W.ru, *rh = r_h ? r_h : W.rh;
    if (!mode_ff(h->prm)) TRY(KL(HDG_PROF_RECOVER, 1, launch_recover(h, ru, rh, lam, u, h_out)));
    else TRY(KL(HDG_PROF_RECOVER, 1, launch_recover_ff(h, ru, rh, lam, u, h_out)));
    return HDG_OK;
}

int hdg_recover(hdg_handle *h, const double *r_u, const double *r_h, const double *lambda, double *u, double *h_out) {
    int rc = require_condensed(h);
    if (rc) return rc;
    if (!u || !h_out) return fail(h, HDG_EINVAL, "NULL output pointer");
    if (!r_u != !r_h) return fail(h, HDG_EINVAL, "r_u and r_h must both be given or both be NULL");
    rc = ensure_staging(h);
    if (rc) return rc;
    Workspace &W = *h->ws;
    cudaStream_t s = h->stream;
    // explicit inputs never overwrite the last solve's right-hand side, which a
    // later call with r_u = r_h = NULL still selects
    const double *ru = W.ru, *rh = W.rh;
    if (r_u) {
        const double *ru_a = host_alias(r_u), *rh_a = host_alias(r_h);
        if (mode_ff(h->prm) && ru_a && rh_a) {
            ru = ru_a;
            rh = rh_a;
        } else {
            if (!W.ru_x) {
                TRY(dalloc(&W.ru_x, size_t(h->N) * 2 * h->np));
                TRY(dalloc(&W.rh_x, size_t(h->N) * h->np));
            }
            TRY(cudaMemcpyAsync(W.ru_x, r_u, sizeof(double) * size_t(h->N) * 2 * h->np, cudaMemcpyHostToDevice, s));
            TRY(cudaMemcpyAsync(W.rh_x, r_h, sizeof(double) * size_t(h->N) * h->np, cudaMemcpyHostToDevice, s));
            ru = W.ru_x;
            rh = W.rh_x;
        }
    } else if (!W.have_z && !W.have_rhs) {
        return fail(h, HDG_ESTATE, "no right-hand side given and none kept from the last solve");
    }
    // the last solve's right-hand side as z_K = R_M r_K kept by its step 1
    const bool from_z = !r_u && W.have_z;
    const double *lam = W.lam_int;
    if (lambda) {
        TRY(cudaMemcpyAsync(W.lam_ext, lambda, sizeof(double) * W.NT, cudaMemcpyHostToDevice, s));
        TRY(KL(HDG_PROF_LAYOUT, 1, launch_to_internal(h, W.lam_ext, W.k64.res)));
        lam = W.k64.res;
    } else if (!W.have_lambda) {
        return fail(h, HDG_ESTATE, "no lambda given and no previous solve");
    }
    double *u_a = host_alias(u), *h_a = host_alias(h_out);
    if (mode_ff(h->prm) && u_a && h_a) {
        // page-locked outputs of a mixed handle: the recovery kernel writes them in place
        if (from_z) TRY(KL(HDG_PROF_RECOVER, 1, launch_recover_z(h, W.z2, lam, u_a, h_a)));
        else TRY(KL(HDG_PROF_RECOVER, 1, launch_recover_ff(h, ru, rh, lam, u_a, h_a)));
    } else {
        if (from_z) TRY(KL(HDG_PROF_RECOVER, 1, launch_recover_z(h, W.z2, lam, W.u, W.hh)));
        else if (!mode_ff(h->prm)) TRY(KL(HDG_PROF_RECOVER, 1, launch_recover(h, ru, rh, lam, W.u, W.hh)));
        else TRY(KL(HDG_PROF_RECOVER, 1, launch_recover_ff(h, ru, rh, lam, W.u, W.hh)));
        TRY(cudaMemcpyAsync(u, W.u, sizeof(double) * size_t(h->N) * 2 * h->np, cudaMemcpyDeviceToHost, s));
        TRY(cudaMemcpyAsync(h_out, W.hh, sizeof(double) * size_t(h->N) * h->np, cudaMemcpyDeviceToHost, s));
    }
    TRY(cudaStreamSynchronize(s));
    return HDG_OK;
}

int hdg_trace_apply_dev(hdg_handle *h, const double *x, double *y) {
    int rc = require_condensed(h);
    if (rc) return rc;
    Workspace &W = *h->ws;
    TRY(KL(HDG_PROF_LAYOUT, 1, launch_to_internal(h, x, W.k64.t0)));
    TRY(KL(HDG_PROF_APPLY64, 1, launch_apply_t<double>(h, W.k64.t0, W.k64.t1)));
    TRY(KL(HDG_PROF_LAYOUT, 1, launch_to_external(h, W.k64.t1, y)));
    return HDG_OK;
}

int hdg_condensed_rhs_dev(hdg_handle *h, const double *r_u, const double *r_h, double *g) {
    int rc = require_condensed(h);
    if (rc) return rc;
    Workspace &W = *h->ws;
    TRY(KL(HDG_PROF_RHS, 2, launch_rhs(h, r_u, r_h, W.g, W.ycell)));
    TRY(KL(HDG_PROF_LAYOUT, 1, launch_to_external(h, W.g, g)));
    return HDG_OK;
}

int hdg_precond_apply_dev(hdg_handle *h, const double *v, double *z) {
    int rc = require_condensed(h);
    if (rc) return rc;
    Workspace &W = *h->ws;
    TRY(KL(HDG_PROF_LAYOUT, 1, launch_to_internal(h, v, W.r)));
    TRY(precond<double>(h, W.r, W.x));
    TRY(KL(HDG_PROF_LAYOUT, 1, launch_to_external(h, W.x, z)));
    return HDG_OK;
}

int hdg_precond_apply32_dev(hdg_handle *h, const float *v, float *z) {
    int rc = require_condensed(h);
    if (rc) return rc;
    if (h->prm.precision == HDG_FP64) return fail(h, HDG_EINVAL, "the FP32 preconditioner needs a mixed precision mode");
    if (!v || !z) return fail(h, HDG_EINVAL, "NULL pointer argument");
    Workspace &W = *h->ws;
    const size_t NF = h->NF, pp = h->pp;
    // [NF][pp] <-> [pp][NF] through the FP32 Krylov work vectors
    TRY(launch_to_internal32(h, v, W.k32.b));
    TRY(precond<float>(h, W.k32.b, W.k32.x));
    (void)NF;
    (void)pp;
    TRY(launch_to_external32(h, W.k32.x, z));
    return HDG_OK;
}

int hdg_get_sizes(const hdg_handle *h, int64_t *sizes) {
    if (!h || !sizes) return HDG_EINVAL;
    sizes[0] = h->N;
    sizes[1] = h->NF;
    sizes[2] = h->NT;
    sizes[3] = h->np;
    sizes[4] = h->m;
    sizes[5] = int64_t(h->lev.size());
    return HDG_OK;
}

int hdg_get_facets(const hdg_handle *h, int32_t *facet_of, int32_t *flip, int32_t *facet_verts) {
    if (!h) return HDG_EINVAL;
    if (facet_of) std::memcpy(facet_of, h->hm.facet_of.data(), sizeof(int32_t) * h->hm.facet_of.size());
    if (flip) std::memcpy(flip, h->hm.flip.data(), sizeof(int32_t) * h->hm.flip.size());
    if (facet_verts) std::memcpy(facet_verts, h->hm.facet_verts.data(), sizeof(int32_t) * h->hm.facet_verts.size());
    return HDG_OK;
}

int hdg_get_cell_schur(hdg_handle *h, double *S) {
    int rc = require_condensed(h);
    if (rc) return rc;
    if (!S) return fail(h, HDG_EINVAL, "NULL output pointer");
    TRY(cudaMemcpyAsync(S, h->d_Scell, sizeof(double) * size_t(h->N) * h->m * h->m, cudaMemcpyDeviceToHost,
                        h->stream));
    TRY(cudaStreamSynchronize(h->stream));
    return HDG_OK;
}

int hdg_profile_enable(hdg_handle *h, int timing_on) {
    if (!h) return HDG_EINVAL;
    if (timing_on < 0 || timing_on > 2) return fail(h, HDG_EINVAL, "timing_on must be 0, 1 or 2");
    TRY(cudaStreamSynchronize(h->stream));
    prof_flush(h);
    Prof &P = h->prof;
    if (timing_on == 2 && !P.evict_buf) {
        int dev = 0, l2 = 0;
        TRY(cudaGetDevice(&dev));
        TRY(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
        P.evict_bytes = (size_t(3) * size_t(l2) + 15) / 16 * 16;
        TRY(cudaMalloc(&P.evict_buf, P.evict_bytes));
        TRY(cudaMalloc(reinterpret_cast<void **>(&P.evict_sink), sizeof(uint32_t)));
        TRY(cudaMemsetAsync(P.evict_buf, 0x5a, P.evict_bytes, h->stream));
        TRY(cudaStreamSynchronize(h->stream));
    } else if (timing_on != 2 && P.evict_buf) {
        cudaFree(P.evict_buf);
        cudaFree(P.evict_sink);
        P.evict_buf = nullptr;
        P.evict_sink = nullptr;
        P.evict_bytes = 0;
    }
    h->prof.on = timing_on != 0;
    for (int i = 0; i < HDG_PROF_N; ++i) {
        h->prof.ms[i] = 0.0;
        h->prof.launches[i] = 0;
    }
    return HDG_OK;
}

int hdg_profile_read(hdg_handle *h, double *ms, int64_t *launches) {
    if (!h) return HDG_EINVAL;
    TRY(cudaStreamSynchronize(h->stream));
    prof_flush(h);
    for (int i = 0; i < HDG_PROF_N; ++i) {
        if (ms) ms[i] = h->prof.ms[i];
        if (launches) launches[i] = h->prof.launches[i];
    }
    return HDG_OK;
}

int hdg_autotune(hdg_handle *h, int32_t *choice) {
    int rc = require_condensed(h);
    if (rc) return rc;
    if (h->prm.flux == 1) return fail(h, HDG_EINVAL, "hdg_autotune serves the upwind solver");
    Workspace &W = *h->ws;
    cudaStream_t s = h->stream;
    const bool f32 = mode_ff(h->prm);   // the Krylov space the Arnoldi steps run in
    const size_t ld = W.ld;
    const int jt = std::min(4, W.m - 1);
    // basis vectors with arbitrary finite content for timing
    if (f32) {
        TRY(launch_fill<float>(W.k32.V, 1.0f, ld * size_t(jt + 2), s));
    } else {
        TRY(launch_fill<double>(W.k64.V, 1.0, ld * size_t(jt + 2), s));
    }
    const bool was_on = h->prof.on;
    h->prof.on = false;
    cudaEvent_t e0, e1;
    TRY(cudaEventCreate(&e0));
    TRY(cudaEventCreate(&e1));
    // time of one Arnoldi step (preconditioner, operator, Gram-Schmidt), best of 3
    auto time_step = [&](float &best) -> int {
        best = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
            TRY(cudaEventRecord(e0, s));
            cudaError_t e = f32 ? arnoldi_step<float>(h, jt) : arnoldi_step<double>(h, jt);
            if (e != cudaSuccess) return fail(h, HDG_ECUDA, std::string("autotune: ") + cudaGetErrorString(e));
            TRY(cudaEventRecord(e1, s));
            TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            TRY(cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0) best = std::min(best, ms);
        }
        return HDG_OK;
    };
    float t;
    // threads per block of the facet-row kernels
    int best_bs = h->bs_facet;
    float best_t = 1e30f;
    for (int bs : {64, 128, 256}) {
        h->bs_facet = bs;
        if ((rc = time_step(t))) return rc;
        if (t < best_t) { best_t = t; best_bs = bs; }
    }
    h->bs_facet = best_bs;
    // blocks of the fused Gram-Schmidt kernels
    int best_nb = W.nblk_gs;
    best_t = 1e30f;
    for (int nb : {152, 304, 608, kMaxGsBlocks}) {
        W.nblk_gs = nb;
        if ((rc = time_step(t))) return rc;
        if (t < best_t) { best_t = t; best_nb = nb; }
    }
    W.nblk_gs = best_nb;
    // first level of the single-CTA coarse cycle
    int best_tm = f32 ? kTailMaxVertices : kTailMaxVertices64;
    best_t = 1e30f;
    int last_ts = -1;
    for (int tm : {256, 1024, 4096}) {
        if ((rc = set_tail_start(h, f32 ? kTailMaxVertices64 : tm, f32 ? tm : kTailMaxVertices))) return rc;
        const int ts = h->tail_start[f32 ? 1 : 0];
        if (ts == last_ts) continue;
        last_ts = ts;
        if ((rc = time_step(t))) return rc;
        if (t < best_t) { best_t = t; best_tm = tm; }
    }
    if ((rc = set_tail_start(h, f32 ? kTailMaxVertices64 : best_tm, f32 ? best_tm : kTailMaxVertices))) return rc;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->prof.on = was_on;
    drop_graphs(h);
    // the timing filled basis vectors over their padded length; the padding
    // beyond N_T must be zero again for the Gram-Schmidt kernels
    if (f32) {
        TRY(cudaMemsetAsync(W.k32.V, 0, sizeof(float) * ld * size_t(W.m + 1), s));
    } else {
        TRY(cudaMemsetAsync(W.k64.V, 0, sizeof(double) * ld * size_t(W.m + 1), s));
    }
    if (choice) {
        choice[0] = h->bs_facet;
        choice[1] = W.nblk_gs;
        choice[2] = h->lev[h->tail_start[f32 ? 1 : 0]].nv;
    }
    return HDG_OK;
}

int hdg_solve_batch_dev(hdg_handle *const *hs, int n, const double *const *r_u, const double *const *r_h,
                        double *const *lambda, hdg_solve_info *infos, int n_threads) {
    if (n < 0 || (n > 0 && (!hs || !r_u || !r_h || !lambda))) return fail(nullptr, HDG_EINVAL, "bad batch arguments");
    for (int i = 0; i < n; ++i) {
        if (!hs[i]) return fail(nullptr, HDG_EINVAL, "NULL handle in the batch");
        for (int j = 0; j < i; ++j)
            if (hs[j] == hs[i] || hs[j]->stream == hs[i]->stream)
                return fail(nullptr, HDG_EINVAL, "batch handles must be distinct and use distinct streams");
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(nullptr, HDG_ECUDA, "cudaGetDevice failed");
    const int nt = std::max(1, std::min(n_threads > 0 ? n_threads : 16, n));
    std::atomic<int> next(0);
    std::vector<int> rcs(size_t(std::max(n, 1)), HDG_OK);
    auto worker = [&]() {
        cudaSetDevice(dev);
        for (;;) {
            const int i = next.fetch_add(1);
            if (i >= n) break;
            hdg_solve_info info{};
            rcs[i] = hdg_solve_dev(hs[i], r_u[i], r_h[i], lambda[i], &info);
            if (infos) infos[i] = info;
        }
    };
    std::vector<std::thread> pool;
    for (int t2 = 1; t2 < nt; ++t2) pool.emplace_back(worker);
    worker();
    for (auto &th : pool) th.join();
    for (int i = 0; i < n; ++i)
        if (rcs[i] != HDG_OK) {
            g_setup_error = "batch entry " + std::to_string(i) + ": " + hs[i]->err;
            return rcs[i];
        }
    return HDG_OK;
}

int hdg_batch_create(hdg_handle *const *hs, int n, hdg_batch **out) {
    if (!out) return fail(nullptr, HDG_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || !hs) return fail(nullptr, HDG_EINVAL, "a batch needs at least one handle");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(nullptr, HDG_ECUDA, "cudaGetDevice failed");
    for (int i = 0; i < n; ++i) {
        hdg_handle *h = hs[i];
        const std::string at = "batch entry " + std::to_string(i) + ": ";
        if (!h) return fail(nullptr, HDG_EINVAL, at + "NULL handle");
        for (int j = 0; j < i; ++j)
            if (hs[j] == h) return fail(nullptr, HDG_EINVAL, at + "the same handle twice");
        if (h->device != dev) return fail(nullptr, HDG_EINVAL, at + "handle set up on another device");
        if (!h->condensed) return fail(nullptr, HDG_ESTATE, at + "hdg_condense has not run on this handle");
        if (!mode_ff(h->prm))
            return fail(nullptr, HDG_EINVAL, at + "merged batches run the precisions HDG_MIXED_FP32 and HDG_MIXED_BF16");
        if (h->prm.flux != 0) return fail(nullptr, HDG_EINVAL, at + "merged batches run the upwind flux");
        if (h->prm.reorth != 0) return fail(nullptr, HDG_EINVAL, at + "merged batches run with reorth = 0");
    }
    std::unique_ptr<hdg_batch, void (*)(hdg_batch *)> b(new hdg_batch, batch_release);
    b->hs.assign(hs, hs + n);
    b->device = dev;
    auto cu = [](cudaError_t e, const char *what) {
        return e == cudaSuccess ? HDG_OK : fail(nullptr, HDG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    };
    int rc;
    // groups: HDG_BATCH_GROUPS = G >= 1 splits the problems, sorted by trace
    // unknowns NT, into G contiguous size classes of about equal total NT (or,
    // with HDG_BATCH_DEAL=rr, deals them round robin); 0 groups them by degree p
    int G = 4;
    if (const char *env = std::getenv("HDG_BATCH_GROUPS")) G = std::atoi(env);
    if (G < 0 || G > 64) return fail(nullptr, HDG_EINVAL, "HDG_BATCH_GROUPS must be 0..64");
    b->group_of.assign(size_t(n), 0);
    if (G == 0) {
        std::vector<int> ps;
        for (int i = 0; i < n; ++i)
            if (std::find(ps.begin(), ps.end(), hs[i]->p) == ps.end()) ps.push_back(hs[i]->p);
        std::sort(ps.begin(), ps.end());
        for (int i = 0; i < n; ++i)
            b->group_of[size_t(i)] = int(std::find(ps.begin(), ps.end(), hs[i]->p) - ps.begin());
        G = int(ps.size());
    } else {
        G = std::min(G, n);
        std::vector<int> order(static_cast<size_t>(n));
        for (int i = 0; i < n; ++i) order[size_t(i)] = i;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return hs[x]->NT > hs[y]->NT; });
        const char *deal = std::getenv("HDG_BATCH_DEAL");
        if (!(deal && std::strcmp(deal, "rr") == 0)) {
            // contiguous size classes of about equal total trace unknowns, so that
            // the problems merged into one launch are of similar size
            double total = 0.0;
            for (int i = 0; i < n; ++i) total += double(hs[i]->NT);
            double acc = 0.0;
            int g = 0;
            for (int k = 0; k < n; ++k) {
                const int i = order[size_t(k)];
                b->group_of[size_t(i)] = g;
                acc += double(hs[i]->NT);
                if (g + 1 < G && acc >= total * double(g + 1) / G && n - k - 1 >= G - g - 1) ++g;
            }
            G = g + 1;
        } else {
            for (int k = 0; k < n; ++k) b->group_of[size_t(order[size_t(k)])] = k % G;
        }
    }
    for (int g = 0; g < G; ++g) {
        std::unique_ptr<hdg_batch::Group> grp(new hdg_batch::Group);
        if ((rc = cu(cudaStreamCreateWithFlags(&grp->stream, cudaStreamNonBlocking), "cudaStreamCreateWithFlags")))
            return rc;
        if ((rc = cu(cudaEventCreateWithFlags(&grp->ev, cudaEventDisableTiming), "cudaEventCreateWithFlags"))) return rc;
        b->groups.push_back(std::move(grp));
    }
    for (int i = 0; i < n; ++i) b->groups[size_t(b->group_of[size_t(i)])]->idx.push_back(i);
    b->ev_in.assign(size_t(n), nullptr);
    for (auto &e : b->ev_in)
        if ((rc = cu(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreateWithFlags"))) return rc;
    if ((rc = cu(cudaMallocHost(reinterpret_cast<void **>(&b->status_host), sizeof(int32_t) * size_t(n)),
                 "cudaMallocHost")))
        return rc;
    std::memset(b->status_host, 0, sizeof(int32_t) * size_t(n));
    if ((rc = cu(cudaHostGetDevicePointer(reinterpret_cast<void **>(&b->status_dev), b->status_host, 0),
                 "cudaHostGetDevicePointer")))
        return rc;
    for (int i = 0; i < n; ++i) {
        std::unique_ptr<Fiber> f(new Fiber);
        f->stack.reset(new unsigned char[kFiberStack]);
        f->status_dev = b->status_dev + i;
        b->fibers.push_back(std::move(f));
    }
    *out = b.release();
    return HDG_OK;
}

int hdg_batch_solve_dev(hdg_batch *b, const double *const *r_u, const double *const *r_h, double *const *lambda,
                        hdg_solve_info *infos) {
    if (!b) return fail(nullptr, HDG_EINVAL, "batch is NULL");
    if (!r_u || !r_h || !lambda) return fail(nullptr, HDG_EINVAL, "NULL pointer argument");
    if (batch_recorder() || t_sched) return fail(nullptr, HDG_ESTATE, "a batched solve is already running on this thread");
    const int n = int(b->hs.size());
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device)
        return fail(nullptr, HDG_EINVAL, "the batch's device is not the current device");
    for (int i = 0; i < n; ++i) {
        hdg_handle *h = b->hs[i];
        const std::string at = "batch entry " + std::to_string(i) + ": ";
        if (!r_u[i] || !r_h[i] || !lambda[i]) return fail(nullptr, HDG_EINVAL, at + "NULL pointer argument");
        if (!h->condensed) return fail(nullptr, HDG_ESTATE, at + "hdg_condense has not run on this handle");
        if (!mode_ff(h->prm) || h->prm.flux != 0 || h->prm.reorth != 0)
            return fail(nullptr, HDG_ESTATE, at + "the handle's parameters changed since hdg_batch_create");
        if (h->prof.on) return fail(nullptr, HDG_ESTATE, at + "kernel timing is on (hdg_profile_enable)");
        if (h->lc.on || h->lc.collecting) return fail(nullptr, HDG_ESTATE, at + "the learned smoother is enabled");
    }
    // each group's stream after the work already queued on its handles' streams
    for (int i = 0; i < n; ++i) {
        cudaError_t e = cudaEventRecord(b->ev_in[size_t(i)], b->hs[size_t(i)]->stream);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(b->groups[size_t(b->group_of[size_t(i)])]->stream, b->ev_in[size_t(i)], 0);
        if (e != cudaSuccess) return fail(nullptr, HDG_ECUDA, std::string("ordering the batch: ") + cudaGetErrorString(e));
    }
    ucontext_t sched;
    for (int i = 0; i < n; ++i) {
        Fiber &f = *b->fibers[size_t(i)];
        f.h = b->hs[size_t(i)];
        f.r_u = r_u[i];
        f.r_h = r_h[i];
        f.lambda = lambda[i];
        f.info = hdg_solve_info{};
        f.rc = HDG_OK;
        f.done = false;
        f.rec.clear();
        b->status_host[i] = 0;
        if (getcontext(&f.ctx) != 0) return fail(nullptr, HDG_EINVAL, "getcontext failed");
        f.ctx.uc_stack.ss_sp = f.stack.get();
        f.ctx.uc_stack.ss_size = kFiberStack;
        f.ctx.uc_link = &sched;
        makecontext(&f.ctx, fiber_entry, 0);
    }
    t_sched = &sched;
    t_wave_error = nullptr;
    std::string wave_err;
    auto set_error = [&](const std::string &m) {
        if (t_wave_error) return;
        wave_err = m;
        t_wave_error = wave_err.c_str();
    };
    // Round-robin over the groups.  In each: resume the fibers whose awaited
    // word has arrived (or that have not started); once none of its fibers
    // waits on a launched wave any more, launch what they recorded as the
    // group's next wave.  A finished wave whose awaited words did not all
    // arrive, or any CUDA error, fails the batch: every fiber is then resumed
    // with the error and unwinds.
    for (auto &g : b->groups) g->inflight = false;
    for (auto &f : b->fibers) {
        f->launched = true;            // not started: resumed on the first pass
        f->wait_addr = nullptr;
    }
    auto resume = [&](Fiber &f) {
        t_fiber = &f;
        batch_recorder() = &f.rec;
        swapcontext(&sched, &f.ctx);
        batch_recorder() = nullptr;
        t_fiber = nullptr;
    };
    for (;;) {
        bool all_done = true;
        for (auto &gp : b->groups) {
            hdg_batch::Group &g = *gp;
            const int64_t t0 = now_ns();
            bool waiting = false;      // some fiber waits on a launched wave
            bool gdone = true;
            for (int i : g.idx) {
                Fiber &f = *b->fibers[size_t(i)];
                if (f.done) continue;
                if (f.launched && (t_wave_error || !f.wait_addr || *f.wait_addr == f.wait_want)) resume(f);
                if (!f.done) {
                    gdone = false;
                    if (f.launched) waiting = true;
                }
            }
            if (waiting && g.inflight && !t_wave_error) {
                // is the last wave over?  then the awaited words must be there
                const cudaError_t q = cudaEventQuery(g.ev);
                if (q == cudaSuccess) {
                    g.inflight = false;
                    std::atomic_thread_fence(std::memory_order_acquire);
                    bool late = false;
                    for (int i : g.idx) {
                        Fiber &f = *b->fibers[size_t(i)];
                        if (!f.done && f.launched && f.wait_addr && *f.wait_addr != f.wait_want) late = true;
                    }
                    if (late) set_error("a wave finished without the value a problem waits for");
                } else if (q != cudaErrorNotReady) {
                    set_error(cudaGetErrorString(q));
                }
            }
            const int64_t t1 = now_ns();
            b->ns_fibers += t1 - t0;
            if (t_wave_error) {
                // nothing more is launched; resume every fiber until it has unwound
                for (int i : g.idx) {
                    Fiber &f = *b->fibers[size_t(i)];
                    f.rec.clear();
                    f.launched = true;
                }
                if (!gdone) all_done = false;
                continue;
            }
            if (!waiting) {
                size_t nrec = 0;
                g.recs.clear();
                for (int i : g.idx) {
                    g.recs.push_back(&b->fibers[size_t(i)]->rec);
                    nrec += b->fibers[size_t(i)]->rec.recs.size();
                }
                if (nrec > 0) {
                    cudaError_t e = g.runner.run(g.recs.data(), int(g.recs.size()), g.stream);
                    if (e == cudaSuccess) e = cudaEventRecord(g.ev, g.stream);
                    if (e == cudaSuccess) g.inflight = true;
                    else set_error(cudaGetErrorString(e));
                    for (int i : g.idx) {
                        Fiber &f = *b->fibers[size_t(i)];
                        f.rec.clear();
                        f.launched = true;
                    }
                } else if (!gdone) {
                    set_error("every problem waits and no launch was recorded");
                }
                b->ns_launch += now_ns() - t1;
            }
            if (!gdone) all_done = false;
        }
        if (all_done) break;
    }
    {
        const int64_t t0 = now_ns();
        for (auto &g : b->groups) {
            const cudaError_t e = cudaStreamSynchronize(g->stream);
            if (e != cudaSuccess) set_error(cudaGetErrorString(e));
        }
        b->ns_wait += now_ns() - t0;
    }
    const bool wave_failed = t_wave_error != nullptr;
    t_sched = nullptr;
    t_wave_error = nullptr;
    int first_rc = HDG_OK;
    std::string first_msg;
    for (int i = 0; i < n; ++i) {
        Fiber &f = *b->fibers[size_t(i)];
        hdg_handle *h = f.h;
        if (!wave_failed && f.rc != HDG_ECUDA && (b->status_host[i] & (8 | 16))) {
            f.rc = fail(h, HDG_ETIMEOUT, (b->status_host[i] & 8)
                                             ? "a bounded device-side wait ran out (coarse-cycle staging)"
                                             : "a bounded device-side wait ran out (tensor-core MMA of the learned sweep)");
            cudaMemsetAsync(h->d_status, 0, sizeof(int32_t), h->stream);
        }
        if (wave_failed && f.rc == HDG_OK) f.rc = fail(h, HDG_ECUDA, "batched solve: " + wave_err);
        f.info.status = f.rc;
        if (infos) infos[i] = f.info;
        if (f.rc != HDG_OK && first_rc == HDG_OK) {
            first_rc = f.rc;
            first_msg = "batch entry " + std::to_string(i) + ": " + h->err;
        }
    }
    // every handle's stream after its group's last wave
    cudaError_t e = cudaSuccess;
    for (auto &g : b->groups)
        if (e == cudaSuccess) e = cudaEventRecord(g->ev, g->stream);
    for (int i = 0; i < n && e == cudaSuccess; ++i)
        e = cudaStreamWaitEvent(b->hs[size_t(i)]->stream, b->groups[size_t(b->group_of[size_t(i)])]->ev, 0);
    if (e != cudaSuccess && first_rc == HDG_OK) {
        first_rc = HDG_ECUDA;
        first_msg = std::string("ordering the handles after the batch: ") + cudaGetErrorString(e);
    }
    if (first_rc != HDG_OK) g_setup_error = first_msg;
    return first_rc;
}

int hdg_batch_solve(hdg_batch *b, const double *const *r_u, const double *const *r_h, double *const *lambda,
                    hdg_solve_info *infos) {
    if (!b) return fail(nullptr, HDG_EINVAL, "batch is NULL");
    if (!r_u || !r_h || !lambda) return fail(nullptr, HDG_EINVAL, "NULL pointer argument");
    const int n = int(b->hs.size());
    std::vector<const double *> du(static_cast<size_t>(n)), dh(static_cast<size_t>(n));
    std::vector<double *> dl(static_cast<size_t>(n));
    for (int i = 0; i < n; ++i) {
        hdg_handle *h = b->hs[size_t(i)];
        const std::string at = "batch entry " + std::to_string(i) + ": ";
        if (!r_u[i] || !r_h[i] || !lambda[i]) return fail(nullptr, HDG_EINVAL, at + "NULL pointer argument");
        if (!h->condensed) return fail(nullptr, HDG_ESTATE, at + "hdg_condense has not run on this handle");
        if (ensure_staging(h)) return fail(nullptr, HDG_ECUDA, at + h->err);
        Workspace &W = *h->ws;
        cudaError_t e = cudaMemcpyAsync(W.ru, r_u[i], sizeof(double) * size_t(h->N) * 2 * h->np,
                                        cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(W.rh, r_h[i], sizeof(double) * size_t(h->N) * h->np, cudaMemcpyHostToDevice,
                                h->stream);
        if (e != cudaSuccess) return fail(nullptr, HDG_ECUDA, at + "staging copy: " + cudaGetErrorString(e));
        du[size_t(i)] = W.ru;
        dh[size_t(i)] = W.rh;
        dl[size_t(i)] = W.lam_ext;
    }
    const int rc = hdg_batch_solve_dev(b, du.data(), dh.data(), dl.data(), infos);
    if (rc == HDG_ECUDA) return rc;
    const std::string msg = rc ? g_setup_error : std::string();
    for (int i = 0; i < n; ++i) {
        hdg_handle *h = b->hs[size_t(i)];
        Workspace &W = *h->ws;
        cudaError_t e = cudaMemcpyAsync(lambda[i], W.lam_ext, sizeof(double) * W.NT, cudaMemcpyDeviceToHost,
                                        h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess)
            return fail(nullptr, HDG_ECUDA, "batch entry " + std::to_string(i) + ": " + cudaGetErrorString(e));
        W.have_rhs = true;   // hdg_recover with NULL right-hand sides uses this solve's
    }
    if (rc) g_setup_error = msg;
    return rc;
}

int hdg_batch_stats(const hdg_batch *b, int64_t *stats) {
    if (!b || !stats) return fail(nullptr, HDG_EINVAL, "NULL pointer argument");
    for (int k = 0; k < 8; ++k) stats[k] = 0;
    for (const auto &g : b->groups) {
        const WaveRunner::Stats &s = g->runner.stats;
        stats[0] += s.waves;
        stats[1] += s.nodes;
        stats[2] += s.records;
        stats[3] += s.hits;
        stats[4] += s.misses;
    }
    stats[5] = b->ns_fibers;
    stats[6] = b->ns_launch;
    stats[7] = b->ns_wait;
    return HDG_OK;
}

int hdg_batch_destroy(hdg_batch *b) {
    if (!b) return HDG_OK;
    for (auto &g : b->groups) cudaStreamSynchronize(g->stream);
    batch_release(b);
    return HDG_OK;
}

void *hdg_get_stream(const hdg_handle *h) { return h ? static_cast<void *>(h->stream) : nullptr; }

// ---------------------------------------------------------------- learned smoother

static uint64_t splitmix64(uint64_t &x) {
    uint64_t z = (x += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

int hdg_learned_init(hdg_handle *h, int hidden, int capacity, uint64_t seed, int32_t *n_params) {
    int rc = require_condensed(h);
    if (rc) return rc;
    if (!mode_ff(h->prm) || !h->d_Sval32)
        return fail(h, HDG_EINVAL, "the learned smoother works in the FP32 inner solves: use HDG_MIXED_FP32 or HDG_MIXED_BF16");
    if (hidden != 32 && hidden != 64) return fail(h, HDG_EINVAL, "hidden width must be 32 or 64");
    if (capacity < 1) return fail(h, HDG_EINVAL, "capacity must be positive");
    Learned &L = h->lc;
    if (L.ready) return fail(h, HDG_ESTATE, "learned smoother already initialised on this handle");
    cudaStream_t s = h->stream;
    const size_t NF = h->NF, NT = h->NT, pp = h->pp, F = 5 * pp;
    L.hid = hidden;
    L.npar = learned_n_params(h->p, hidden);
    L.cap = capacity;
    TRY(dalloc(&L.theta, size_t(L.npar)));
    TRY(dalloc(&L.wimg, learned_tc_image_elems(h->p, hidden)));
    TRY(dalloc(&L.m, size_t(L.npar)));
    TRY(dalloc(&L.v, size_t(L.npar)));
    TRY(dalloc(&L.grad, size_t(L.npar)));
    TRY(dalloc(&L.act, NF * (F + 2 * hidden + 1)));
    TRY(dalloc(&L.gfac, NF * (2 * hidden + pp)));
    TRY(dalloc(&L.gpart, (NF + 1023) / 1024 * size_t(L.npar)));
    TRY(dalloc(&L.rev, 4 * NF));
    TRY(dalloc(&L.buf, size_t(capacity) * NT));
    TRY(dalloc(&L.c, NT));
    TRY(dalloc(&L.rn, NT));
    TRY(dalloc(&L.gc, NT));
    TRY(dalloc(&L.tmp, NT));
    TRY(dalloc(&L.coef, 1));
    TRY(dalloc(&L.nrm, 1));
    TRY(cudaMemsetAsync(L.m, 0, sizeof(float) * L.npar, s));
    TRY(cudaMemsetAsync(L.v, 0, sizeof(float) * L.npar, s));
    // reverse neighbour lists for S^T: facet e appears in the row of each of its
    // four neighbours f, as block b
    std::vector<int32_t> nbr(4 * NF), rev(4 * NF, -1);
    TRY(cudaMemcpyAsync(nbr.data(), h->d_nbr, sizeof(int32_t) * nbr.size(), cudaMemcpyDeviceToHost, s));
    TRY(cudaStreamSynchronize(s));
    std::vector<int> fill(NF, 0);
    for (size_t f = 0; f < NF; ++f)
        for (int b = 1; b <= 4; ++b) {
            const int e = nbr[size_t(b - 1) * NF + f];
            if (fill[e] >= 4) return fail(h, HDG_EINVAL, "facet neighbour relation is not symmetric");
            rev[size_t(fill[e]++) * NF + e] = int32_t(f) * 8 + b;
        }
    for (size_t e = 0; e < NF; ++e)
        if (fill[e] != 4) return fail(h, HDG_EINVAL, "facet neighbour relation is not symmetric");
    TRY(cudaMemcpyAsync(L.rev, rev.data(), sizeof(int32_t) * rev.size(), cudaMemcpyHostToDevice, s));
    // weights: uniform(-a, a) with a = sqrt(3 / fan_in); the output layer 100x
    // smaller and zero biases, so the untrained sweep is close to block-Jacobi
    std::vector<float> th(size_t(L.npar), 0.f);
    uint64_t st = seed;
    auto uni = [&]() { return float((splitmix64(st) >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0); };
    const int hid = hidden;
    size_t k = 0;
    for (size_t i = 0; i < size_t(hid) * F; ++i) th[k++] = uni() * std::sqrt(3.f / float(F));
    k += hid;
    for (size_t i = 0; i < size_t(hid) * hid; ++i) th[k++] = uni() * std::sqrt(3.f / float(hid));
    k += hid;
    for (size_t i = 0; i < pp * size_t(hid); ++i) th[k++] = 0.01f * uni() * std::sqrt(3.f / float(hid));
    TRY(cudaMemcpyAsync(L.theta, th.data(), sizeof(float) * th.size(), cudaMemcpyHostToDevice, s));
    TRY(launch_learned_tc_weights(h));
    TRY(cudaStreamSynchronize(s));
    L.rng = seed ^ 0x5851f42d4c957f2dull;
    L.t = 0;
    L.count = 0;
    L.ready = true;
    if (n_params) *n_params = L.npar;
    return HDG_OK;
}

int hdg_learned_collect_dev(hdg_handle *h, const double *r_u, const double *r_h, int32_t *n_stored) {
    int rc = require_condensed(h);
    if (rc) return rc;
    if (!h->lc.ready) return fail(h, HDG_ESTATE, "hdg_learned_init has not run");
    const bool was_on = h->lc.on;
    h->lc.on = false;
    h->lc.collecting = true;
    hdg_solve_info info{};
    rc = solve_internal(h, r_u, r_h, info);
    h->lc.collecting = false;
    h->lc.on = was_on;
    if (n_stored) *n_stored = h->lc.count;
    return rc;
}

int hdg_learned_train(hdg_handle *h, int steps, int batch, double lr, double *loss_first, double *loss_last) {
    int rc = require_condensed(h);
    if (rc) return rc;
    Learned &L = h->lc;
    if (!L.ready || L.count < 1) return fail(h, HDG_ESTATE, "no training residuals collected");
    if (steps < 1 || batch < 1 || !(lr > 0)) return fail(h, HDG_EINVAL, "bad training arguments");
    Workspace &W = *h->ws;
    cudaStream_t s = h->stream;
    const size_t NT = h->NT;
    W.host_buf[5] = -2.0 / batch;          // stored residuals have unit norm
    TRY(cudaMemcpyAsync(L.coef, W.host_buf + 5, sizeof(double), cudaMemcpyHostToDevice, s));
    for (int step = 0; step < steps; ++step) {
        TRY(cudaMemsetAsync(L.grad, 0, sizeof(float) * L.npar, s));
        double loss = 0.0;
        for (int b = 0; b < batch; ++b) {
            const float *r = L.buf + size_t(splitmix64(L.rng) % uint64_t(L.count)) * NT;
            TRY(launch_learned_forward(h, r, L.c));
            TRY(launch_residual_t<float>(h, r, L.c, L.rn, false));
            double nrn;
            rc = norm_host<float>(h, L.rn, nrn);
            if (rc) return rc;
            loss += nrn * nrn;
            TRY(launch_learned_applyT(h, L.rn, L.gc));
            TRY(launch_learned_backward(h, L.gc, L.coef));
        }
        L.t += 1;
        TRY(launch_adam(h, float(lr), int(std::min<long long>(L.t, 1 << 30))));
        TRY(launch_learned_tc_weights(h));
        loss /= batch;
        if (!std::isfinite(loss)) return fail(h, HDG_ENAN, "NaN in the training loss");
        if (step == 0 && loss_first) *loss_first = loss;
        if (loss_last) *loss_last = loss;
    }
    TRY(cudaStreamSynchronize(s));
    return HDG_OK;
}

int hdg_learned_params(hdg_handle *h, float *theta, int get) {
    if (!h) return HDG_EINVAL;
    if (!h->lc.ready) return fail(h, HDG_ESTATE, "hdg_learned_init has not run");
    if (!theta) return fail(h, HDG_EINVAL, "NULL pointer argument");
    const size_t bytes = sizeof(float) * h->lc.npar;
    if (get) TRY(cudaMemcpyAsync(theta, h->lc.theta, bytes, cudaMemcpyDeviceToHost, h->stream));
    else {
        TRY(cudaMemcpyAsync(h->lc.theta, theta, bytes, cudaMemcpyHostToDevice, h->stream));
        TRY(launch_learned_tc_weights(h));
    }
    TRY(cudaStreamSynchronize(h->stream));
    return HDG_OK;
}

int hdg_learned_enable(hdg_handle *h, int on) {
    if (!h) return HDG_EINVAL;
    if (on < 0 || on > 2) return fail(h, HDG_EINVAL, "on must be 0, 1 or 2");
    if (on && !h->lc.ready) return fail(h, HDG_ESTATE, "hdg_learned_init has not run");
    // the choice of inference kernel is baked into the captured Arnoldi steps
    if (h->lc.tc != (on == 2)) drop_graphs(h);
    h->lc.on = on != 0;
    h->lc.tc = on == 2;
    return HDG_OK;
}

int hdg_learned_loss_grad_dev(hdg_handle *h, const float *R, int n, float *grad, double *loss) {
    int rc = require_condensed(h);
    if (rc) return rc;
    Learned &L = h->lc;
    if (!L.ready) return fail(h, HDG_ESTATE, "hdg_learned_init has not run");
    if (!R || n < 1) return fail(h, HDG_EINVAL, "bad arguments");
    Workspace &W = *h->ws;
    cudaStream_t s = h->stream;
    const size_t NT = h->NT;
    TRY(cudaMemsetAsync(L.grad, 0, sizeof(float) * L.npar, s));
    double total = 0.0;
    for (int i = 0; i < n; ++i) {
        TRY(launch_to_internal32(h, R + size_t(i) * NT, L.tmp));
        double nr;
        rc = norm_host<float>(h, L.tmp, nr);
        if (rc) return rc;
        W.host_buf[6] = -2.0 / (double(n) * nr * nr);
        TRY(cudaMemcpyAsync(L.coef, W.host_buf + 6, sizeof(double), cudaMemcpyHostToDevice, s));
        TRY(launch_learned_forward(h, L.tmp, L.c));
        TRY(launch_residual_t<float>(h, L.tmp, L.c, L.rn, false));
        double nrn;
        rc = norm_host<float>(h, L.rn, nrn);
        if (rc) return rc;
        total += (nrn * nrn) / (nr * nr) / n;
        TRY(launch_learned_applyT(h, L.rn, L.gc));
        TRY(launch_learned_backward(h, L.gc, L.coef));
        TRY(cudaStreamSynchronize(s));
    }
    if (grad) TRY(cudaMemcpyAsync(grad, L.grad, sizeof(float) * L.npar, cudaMemcpyDeviceToHost, s));
    TRY(cudaStreamSynchronize(s));
    if (loss) *loss = total;
    return HDG_OK;
}

int hdg_destroy(hdg_handle *h) {
    free_handle(h);
    return HDG_OK;
}

const char *hdg_last_error(const hdg_handle *h) {
    return h ? h->err.c_str() : g_setup_error.c_str();
}

}  // extern "C"
