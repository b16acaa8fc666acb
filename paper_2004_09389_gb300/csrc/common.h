// Internal declarations of the HDG trace-solver library (not part of the ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <complex>
#include <cstdint>
#include <cstring>
#include <functional>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "../../include/hdg.h"

namespace hdg {

// ---------------------------------------------------------------- sizes

inline int n_cell_nodes(int p) { return (p + 1) * (p + 2) / 2; }

// ---------------------------------------------------------------- reference element
// Reference triangle (0,0),(1,0),(0,1); Lagrange basis at (a/p, b/p), b outer;
// local edge i from vertex (i+1)%3 to (i+2)%3; trace basis at t_j = j/p.
struct RefElem {
    int p = 0, n = 0, pp = 0;
    std::vector<double> M;        // [n][n]      int phi_a phi_b
    std::vector<double> ML;       // [3][n][n]   int L_i phi_a phi_b
    std::vector<double> Dxi;      // [n][n]      int phi_a d_xi phi_b
    std::vector<double> Deta;     // [n][n]
    std::vector<double> E;        // [3][n][n]   edge i: int_0^1 phi_a phi_b dt
    std::vector<double> N;        // [3][n][pp]  edge i: int_0^1 phi_a mu_j dt
    std::vector<double> M1;       // [pp][pp]    int_0^1 mu_j mu_k dt
    // packed copy for the device: M | ML | Dxi | Deta | E | N | M1
    std::vector<double> packed() const;
};
RefElem build_ref_elem(int p);

// offsets into the packed reference data
struct RefOffsets {
    int M, ML, Dxi, Deta, E, N, M1, total;
};
inline RefOffsets ref_offsets(int p) {
    int n = n_cell_nodes(p), pp = p + 1;
    RefOffsets o;
    o.M = 0; o.ML = o.M + n * n; o.Dxi = o.ML + 3 * n * n; o.Deta = o.Dxi + n * n;
    o.E = o.Deta + n * n; o.N = o.E + 3 * n * n; o.M1 = o.N + 3 * n * pp; o.total = o.M1 + pp * pp;
    return o;
}

// ---------------------------------------------------------------- host mesh data
// Patches of the fused P1 smoothing kernels between a level (fine) and the
// next coarser one.  The coarse vertices are split into nb spatially compact
// patches (recursive coordinate bisection).  Going down, patch b takes its
// coarse vertices' children F0 (slots [0, n0)) and their ELL neighbours (the
// rest of F1); going up, it owns the fine vertices whose first parent is in
// it (slots [0, nown)) plus their neighbours.  Every ELL column of a row in
// the first part maps to a slot of the same patch.
struct HostPatches {
    int nb = 0, max_f1 = 0, max_f0 = 0, max_g1 = 0;
    std::vector<int32_t> f_ptr, f_n0, f_ids, f0_base, lcol;        // down: F1 ids per patch, F0 rows' local columns
    std::vector<int32_t> c_ptr, c_ids, cc_ptr, cc_slot;            // down: coarse vertices, their children's slots
    std::vector<double> cc_w;                                      //       and weights (order of child_idx)
    std::vector<int32_t> g_ptr, g_nown, g_ids, g0_base, glcol;     // up: owned + neighbour ids, owned rows' local columns
    // copies of static structure indexed by patch row (no index indirection in the kernels)
    std::vector<int32_t> fcol;        // [f_ids.size()][W] global columns of the F1 rows
    std::vector<int32_t> gcol;        // [g_ids.size()][W] global columns of the up rows
    std::vector<int32_t> gpar;        // [g_ids.size()][W][2] parents (coarse) of each column
    std::vector<int32_t> grow_par;    // [g_ids.size()][2] parents of the row vertex
};

struct HostLevel {
    int nv = 0, nc = 0;
    int vdim = 0;
    std::vector<double> vxyz;     // [nv][vdim] vertex coordinates (coarse levels)
    HostPatches patch;            // fused-kernel patches towards the next coarser level
    std::vector<double> X;        // [nc][3][2] local 2-D vertex coordinates
    std::vector<int32_t> cells;   // [nc][3]
    // padded row-major ELL structure of the level operator: width W (a multiple
    // of 4), slot q of row v at v * W + q (columns increasing, unused slots
    // point at v with value 0)
    int width = 0;
    std::vector<int32_t> col, diag;     // [W * nv], [nv] (slot of the diagonal)
    std::vector<double> elem;           // [nc][27]: 3x3 mass | stiffness | skew per cell
    std::vector<int32_t> contrib_ptr;   // [W * nv + 1]
    std::vector<int32_t> contrib;       // cell*9 + a*3 + b, in cell order per entry
    // transfer to the next finer level (empty on the fine level)
    std::vector<int32_t> parent;      // [nv_finer][2]
    std::vector<int32_t> child_ptr;   // [nv + 1]  restriction: coarse vertex <- fine vertices
    std::vector<int32_t> child_idx;
    std::vector<double> child_w;
};

struct HostMesh {
    int dim = 0, nv = 0, nc = 0, nf = 0;
    std::vector<double> X;            // [nc][3][2] local 2-D coordinates of the fine cells
    std::vector<int32_t> cells;       // [nc][3]
    std::vector<int32_t> facet_of;    // [nc][3]
    std::vector<int32_t> flip;        // [nc][3]
    std::vector<int32_t> facet_verts; // [nf][2] lo, hi
    std::vector<int32_t> facet_cell;  // [nf][2] incident cells (order of appearance)
    std::vector<int32_t> facet_edge;  // [nf][2] local edge index in each cell
    std::vector<int32_t> v2f_ptr;     // [nv+1] vertex -> incident facet ends
    std::vector<int32_t> v2f;         // 2*facet + (0: lo end, 1: hi end)
    std::vector<HostLevel> levels;    // P1 levels, level 0 = fine mesh
};

// Returns empty string on success, else the reason.
std::string build_host_mesh(const hdg_mesh_desc *desc, HostMesh &hm);
// Patches of level l towards level l + 1 (needs both levels' ELL structure,
// the transfers and level l + 1's coordinates); about target_blocks patches.
void build_p1_patches(HostMesh &hm, int l, int target_blocks);

// ---------------------------------------------------------------- device data
struct DevLevel {
    int nv = 0, nnz = 0, width = 0;                     // nnz = width * nv (padded ELL slots)
    int32_t *col = nullptr, *diag = nullptr;
    double *elem = nullptr, *fK = nullptr, *A = nullptr, *dinv = nullptr;
    int32_t *contrib_ptr = nullptr, *contrib = nullptr;
    float *A32 = nullptr, *dinv32 = nullptr;
    int32_t *parent = nullptr;                         // [nv_finer][2]
    int32_t *child_ptr = nullptr, *child_idx = nullptr;
    double *child_w = nullptr;
    float *child_w32 = nullptr;
    int nci = 0;                                        // restriction entries (children)
    // work vectors
    double *x = nullptr, *x2 = nullptr, *b = nullptr, *r = nullptr;
    float *x32 = nullptr, *x232 = nullptr, *b32 = nullptr, *r32 = nullptr;
    // patches of the fused smoothing kernels towards the next coarser level
    // (HostPatches; nb = 0 on the coarsest level)
    int nb = 0, max_f1 = 0, max_f0 = 0, max_g1 = 0;
    int32_t *pf_ptr = nullptr, *pf_n0 = nullptr, *pf_ids = nullptr, *pf0_base = nullptr, *plcol = nullptr;
    int32_t *pc_ptr = nullptr, *pc_ids = nullptr, *pcc_ptr = nullptr, *pcc_slot = nullptr;
    double *pcc_w = nullptr;
    float *pcc_w32 = nullptr;
    int32_t *pg_ptr = nullptr, *pg_nown = nullptr, *pg_ids = nullptr, *pg0_base = nullptr, *pglcol = nullptr;
    int32_t *pfcol = nullptr, *pgcol = nullptr, *pgpar = nullptr, *pgrow_par = nullptr;
};

struct Workspace;   // solver vectors, defined in api.cu

// learned facet-patch smoother (k_learned.cu; an extension beyond the paper)
struct Learned {
    int hid = 0, npar = 0;
    bool ready = false;        // initialised
    bool on = false;           // used by the FP32 preconditioner
    bool tc = false;           // inference on the tensor cores (BF16 weights, FP32 accumulation)
    __nv_bfloat16 *wimg = nullptr;   // BF16 weight images for the tensor-core inference
    bool suspended = false;    // switched off for the rest of a solve after a stall
    bool collecting = false;   // plain solves store the residual before the last sweep
    bool fallback = false;     // a stall was seen in the current solve
    int cap = 0, count = 0;    // training residuals stored / capacity
    long long t = 0;           // Adam steps done
    uint64_t rng = 0;
    float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    float *act = nullptr, *gfac = nullptr;   // per-facet activations / gradients (training)
    float *gpart = nullptr;                  // per-block partial weight gradients [ceil(NF/1024)][npar]
    int32_t *rev = nullptr;                  // [4][NF] neighbour f*8 + block index pointing back
    float *buf = nullptr;                    // [cap][NT] normalised training residuals
    float *c = nullptr, *rn = nullptr, *gc = nullptr, *tmp = nullptr;
    double *coef = nullptr, *nrm = nullptr;
};

// Galerkin coarse operators (k_galerkin.cu, coarse_mode 2): per ELL slot of
// level 0 the codes e*20 + b*4 + sv*2 + sw of its facet-row contributions;
// per slot of level l+1 the (slot of level l, weight) pairs
struct GalerkinHost {
    std::vector<int32_t> ptr0, code0;
    std::vector<std::vector<int32_t>> ptr, idx;
    std::vector<std::vector<double>> w;
};
struct GalerkinDev {
    int32_t *ptr0 = nullptr, *code0 = nullptr;
    std::vector<int32_t *> ptr, idx;
    std::vector<double *> w;
};
std::string build_galerkin_lists(const HostMesh &hm, GalerkinHost &g);

// RT0 coarse space of the Lax-Friedrichs solver (k_lf.cu): facet-row
// neighbours, prolongation weights piw [(b TB + q) NF + e], the reverse
// neighbour map rev [(b'-1) NF + f], per-cell 3 x 3 matrices [N][M | R | D],
// cell means of f, and per ELL slot (b NF + f) the contribution codes K*9 + i*3 + j
struct Rt0Host {
    std::vector<int32_t> nbr, rev, ptr, code;
    std::vector<double> piw, loc, fK;
};
struct Rt0Dev {
    int32_t *nbr = nullptr, *rev = nullptr, *ptr = nullptr, *code = nullptr;
    double *piw = nullptr, *loc = nullptr, *fK = nullptr;
    double *Sc = nullptr, *dinv = nullptr;       // [5][NF] coarse operator, [NF] inverse diagonal
    double *rc = nullptr, *e0 = nullptr, *e1 = nullptr, *e2 = nullptr;   // coarse vectors
};
std::string build_rt0(const HostMesh &hm, int p, Rt0Host &o);

// IMEX time stepping state (k_imex.cu)
constexpr int kImexMaxStages = 5;
struct Imex {
    bool ready = false;
    bool has_f = false;          // explicit Coriolis term present
    size_t nq = 0;               // doubles of one state vector: N * 3 * n_p (u part, then h part)
    double *fcell = nullptr;     // [N][3] Coriolis at the cell vertices (explicit term)
    double *minv = nullptr;      // [n_p][n_p] inverse of the reference mass matrix
    double *lam = nullptr;       // [PP][NF] upwind trace of the DG state
    double *lam_out = nullptr;   // [NF][PP] trace solution of a stage solve
    double *buf = nullptr;       // (3 + 2 kImexMaxStages) state vectors
};

// per-iteration readback of the Krylov driver (pinned host copy)
// a scalar handed to the host through page-locked memory: the value, then
// (after a system-scope fence) a sequence number the host waits for
struct HostValue {
    double v;
    int32_t seq;
    int32_t pad;
};

struct ReadBack {
    double est;      // |s_{j+1}| / ||b||
    double hnext;    // h_{j+1,j} before rotation
    int32_t flags;   // 2: breakdown, 4: NaN/Inf
    int32_t seq;     // page-locked copy only: j + 1, written last (after the other fields) by step j
};

#ifdef __CUDACC__
// The last block of a grid-wide reduction: out[i] = sum over b < nb of
// partial[i * nb + b] for i < k, in a fixed order.  The warps are shared out
// among the vectors (all of them for one vector, half each for two, ...);
// a warp's lanes take every 32 * (warps per vector)-th partial, then a
// shuffle tree, then the vector's warps in order.  Every thread of the block
// must call it.
__device__ __forceinline__ void finish_partials(const double *partial, int nb, int k, double *out) {
    __shared__ double red[32];
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nwarp = blockDim.x / 32;
    const int wpv = nwarp / k > 1 ? nwarp / k : 1, vpr = nwarp / wpv;
    for (int i0 = 0; i0 < k; i0 += vpr) {
        const int i = i0 + warp / wpv, sub = warp % wpv;
        double v = 0.0;
        if (warp < vpr * wpv && i < k)
            for (int b = sub * 32 + lane; b < nb; b += wpv * 32) v += partial[size_t(i) * nb + b];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) red[warp] = v;
        __syncthreads();
        if (int(threadIdx.x) < vpr && i0 + int(threadIdx.x) < k) {
            double t = 0.0;
            for (int q = 0; q < wpv; ++q) t += red[threadIdx.x * wpv + q];
            out[i0 + threadIdx.x] = t;
        }
        __syncthreads();
    }
}
#endif

// levels of the single-CTA V-cycle tail (k_p1.cu)
constexpr int kMaxGsBlocks = 1216;     // largest grid of the fused Gram-Schmidt kernels (8 x 152 SMs)
constexpr int kTailMaxLevels = 8;
constexpr int kTailMaxVertices = 1024;     // default largest level run inside the tail kernel
constexpr int kTailMaxVertices64 = 256;    // the same for the FP64 levels (measured faster there)
constexpr size_t kTailSmemMax = 226 * 1024; // dynamic shared memory limit of the tail kernel
constexpr size_t kTailInvSmemMax = 64 * 1024; // largest coarsest-level inverse staged in shared memory
constexpr int kPatchMaxVertices = 32768;      // largest P1 level smoothed by the fused patch kernels
// One level of the single-CTA tail as laid out in shared memory: sizes and
// byte offsets from the start of the dynamic shared memory.  The table sits
// at offset 0 of the tail image; arrays that the bulk copy does not fill
// (x, x2, b, r) lie after the image.
struct TailHdr {
    int32_t nv, nnz, nci, W;            // nnz = W * nv; nci = 0 on the first tail level
    int32_t oA, oD, ocw, ocol, ocp, oci, opar;   // staged: values, inverse diagonal, transfers
    int32_t ox, ox2, ob, orr, pad;      // scratch vectors
};
static_assert(sizeof(TailHdr) == 64, "tail header entries are 64 bytes");
// The tail's shared-memory image in global memory for one precision:
// [TailHdr per level][level arrays, each 16-byte padded][coarsest inverse
// when it fits], filled at condensation, staged by bulk copies per launch.
struct TailImage {
    unsigned char *d = nullptr;
    size_t cap = 0;
    int ts = -1;                        // first level the image was built for
    uint32_t img_bytes = 0;             // bytes staged by the bulk copies
    uint32_t smem_bytes = 0;            // image plus scratch vectors
    int32_t inv_off = -1;               // offset of the staged inverse, -1: read from global memory
    int32_t ob0 = 0, ox0 = 0;           // scratch b and x of the first tail level
};
// shared-memory bytes of the tail kernel for levels [first, levels.size()) in
// precision of size tsz (header table, level arrays, scratch; no inverse)
size_t tail_smem_bytes(const std::vector<DevLevel> &lev, int first, size_t tsz);

// Host-side layout of the tail image (csrc/layout.cpp).  Sizes of one tail
// level: vertices, ELL slots and width, restriction entries into it and the
// finer level's vertex count (both 0 on the first tail level).
struct TailLevelSize {
    int nv, nnz, W, nci, nfin;
};
// (kTailA: ELL values slot-major; kTailCol: ELL columns as 16-bit indices)
enum TailPieceKind : int { kTailA = 0, kTailD, kTailCol, kTailCw, kTailCp, kTailCi, kTailPar, kTailInv };
// one array copied into the image: byte offset and (16-byte padded) size,
// the tail level it belongs to and what it is
struct TailPiece {
    size_t off, bytes;
    int level, kind;
};
struct TailLayout {
    std::vector<TailHdr> hdr;         // one per level, at offset 0 of the image
    std::vector<TailPiece> pieces;    // in offset order, after the table
    size_t img_bytes = 0;             // table + pieces: what the bulk copies stage
    size_t smem_bytes = 0;            // plus the scratch vectors x, x2, b, r of every level
    int32_t inv_off = -1;             // offset of the coarsest FP64 inverse, -1: not staged
};
// The layout for levels lv (first tail level first), values of tsz bytes and
// a coarsest level of nc vertices whose FP64 inverse is staged when it fits
// (nc = 0: never).  Every offset and size is a multiple of 16 bytes.  Returns
// false when the shared memory would exceed kTailSmemMax.
bool tail_layout(const std::vector<TailLevelSize> &lv, size_t tsz, size_t nc, TailLayout &out);
struct TailArgs {
    int nlev, nu1, nu2;
    double omega;
    const unsigned char *img;           // tail image (global), 16-byte aligned
    uint32_t img_bytes;                 // bytes to stage, a multiple of 16
    int32_t inv_off;                    // staged inverse offset, -1: use inv
    int32_t nv0, ob0, ox0;              // first tail level: size, scratch offsets of b and x
    const void *dinv0;                  // its inverse diagonal (global, the solve precision)
    int32_t *status;                    // device error flags (8: shared-memory staging timed out)
    const double *inv;                  // dense FP64 inverse of the last level (n x n, row-major)
    const void *b_top;                  // right-hand side of the first tail level (global)
    void *x_top;                        // its solution (global)
};

// ---------------------------------------------------------------- two-float arithmetic
// An FP64 value a as the pair (hi, lo) = (rn(a), rn(a - hi)) of floats; a sum
// of products carried as s + c: s the running sum of the rounded leading
// products, added by error-free TwoSum steps, c the float sum of the exact
// product errors (by FMA), the cross terms and the TwoSum errors.  About
// n * 2^-48 relative error of sum |a_i x_i| for n terms, a dozen FP32
// operations per term (used where GB300's FP64 pipe would be the bound).
__device__ __forceinline__ float2 split(double a) {
    const float hi = __double2float_rn(a);
    return make_float2(hi, __double2float_rn(a - double(hi)));
}

// Cell tiles of the two-float per-cell matrices: a matrix a (rows x cols per
// cell) is stored as pairs of consecutive row entries, (hi, lo) of column 2cp
// and of column 2cp + 1 (zeros past the row's end) in one float4, pair plane
// pc = row * CP + cp (CP = (cols + 1) / 2) of cell K at
// ((K / kFFCells) * rows * CP + pc) * kFFCells + K % kFFCells.
constexpr int kFFCells = 32;
__host__ __device__ __forceinline__ size_t ff_pair_index(size_t K, size_t pc, size_t np) {
    return ((K / kFFCells) * np + pc) * kFFCells + K % kFFCells;
}

struct FFAcc {
    float s = 0.f, c = 0.f;
    // s + c += a * x (a, x split pairs); intrinsics keep the compiler from
    // contracting or reassociating the error-free steps
    __device__ __forceinline__ void add(const float2 a, const float2 x) {
        const float p = __fmul_rn(a.x, x.x);
        const float e = __fmaf_rn(a.x, x.x, -p);
        c = __fmaf_rn(a.x, x.y, c);
        c = __fmaf_rn(a.y, x.x, c);
        c = __fadd_rn(c, e);
        const float t = __fadd_rn(s, p);
        const float bp = __fsub_rn(t, s);
        c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp)));
        s = t;
    }
    __device__ __forceinline__ double value() const { return double(s) + double(c); }
};

// ---------------------------------------------------------------- dependent launch
// Programmatic dependent launch (sm_90 and later): a kernel launched by
// pdl_launch may be scheduled while the previous kernel in the stream drains
// its last blocks, which hides most of the launch and dispatch latency of
// short kernels.  Such a kernel calls pdl_wait() before it touches any global
// memory: the wait returns once the previous kernel has completed and its
// writes are visible (for a kernel launched without the attribute it returns
// at once).  pdl_wait() then lets the next kernel be scheduled in turn.
__device__ __forceinline__ void pdl_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
// Families of kernels launched with the attribute: HDG_PDL is a bit mask (1:
// facet-row kernels, 2: P1 kernels, 4: Krylov and copy kernels; read once).
// The default 6 leaves out the facet-row kernels: measured on the flat
// 256 x 256 x 2, p = 3 mixed-precision solve, the attribute on them cost about
// 5 % of the solve rate, on the P1 and Krylov kernels it gained about 1 %.
bool pdl_enabled(unsigned family);
template <typename... KP, typename... A>
void pdl_launch(unsigned family, void (*k)(KP...), unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                A &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled(family) ? 1 : 0;
    (void)cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);   // errors surface through cudaGetLastError
}

// ---------------------------------------------------------------- merged launches
// A batched solve runs the launch sequences of many independent problems at
// once.  Each kernel that takes part exists in three forms: NAME_impl, the
// body as a device function of (block index, grid size, arguments); NAME, the
// ordinary kernel; and NAME_multi, one launch over several problems, whose
// blocks start[i] .. start[i+1]-1 run problem i's blocks with problem i's
// arguments.  The launch helper NAME_go launches NAME, or, while a Recorder is
// installed on the calling thread, appends a record of the launch instead; the
// batch then merges records of different problems that use the same kernel
// and block size into one NAME_multi launch.  Every argument travels in the
// kernel's parameter block (up to kMergeMax problems per launch).
constexpr int kMergeMax = 64;

template <class A>
struct MultiP {
    int n;                        // problems in this launch
    int start[kMergeMax + 1];     // first block of problem i; start[n] = total blocks
    A a[kMergeMax];               // arguments of problem i
};

// problem of this block (binary search of start) and the block's index within it
__device__ __forceinline__ int merge_find(const int *start, int n, int &local) {
    const int b = int(blockIdx.x);
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    local = b - start[lo];
    return lo;
}

struct MergeRec {
    const void *func;             // the merged kernel (a NAME_multi instantiation)
    void (*pack)(void *out, int n, const int *start, const unsigned char *const *args);
    uint32_t param_bytes;         // sizeof(MultiP<A>)
    uint32_t args_bytes;          // sizeof(A)
    unsigned grid, block;         // this problem's launch shape
    size_t smem;
    size_t off;                   // the arguments, in the recorder's arena
    unsigned family;              // the kernel's launch family (pdl_launch): a merged launch of an
                                  // enabled family depends on its predecessors by programmatic edges
};
struct Recorder {
    std::vector<MergeRec> recs;
    std::vector<unsigned char> arena;
    void clear() {
        recs.clear();
        arena.clear();
    }
};
// the calling thread's recorder (null: launch directly)
Recorder *&batch_recorder();

template <class A>
void merge_pack(void *out, int n, const int *start, const unsigned char *const *args) {
    static_assert(std::is_trivially_copyable<A>::value, "merged-launch arguments are copied bytewise");
    static_assert(sizeof(MultiP<A>) <= 32000, "merged-launch parameters exceed the kernel parameter limit");
    MultiP<A> *M = static_cast<MultiP<A> *>(out);
    std::memset(out, 0, sizeof(MultiP<A>));
    M->n = n;
    for (int i = 0; i <= n; ++i) M->start[i] = start[i];
    for (int i = 0; i < n; ++i) std::memcpy(static_cast<void *>(&M->a[i]), args[i], sizeof(A));
}
// a (built in zeroed storage, so that its padding bytes are zero and two
// records of the same launch compare equal byte for byte)
template <class A>
void batch_record(Recorder *r, const void *func, const A &a, unsigned grid, unsigned block, size_t smem,
                  unsigned family) {
    MergeRec m{func, &merge_pack<A>, uint32_t(sizeof(MultiP<A>)), uint32_t(sizeof(A)), grid, block, smem,
               r->arena.size(), family};
    const unsigned char *p = reinterpret_cast<const unsigned char *>(&a);
    r->arena.insert(r->arena.end(), p, p + sizeof(A));
    r->recs.push_back(m);
}

// stream-ordered copy of n bytes (src null: zero fill) as a kernel, so that a
// batched solve can record it; src may be page-locked host memory
cudaError_t launch_copy(void *dst, const void *src, size_t n, cudaStream_t s);

// One wave of a batched solve: the launches that every problem records
// between two host decisions, merged into NAME_multi launches and run as a
// CUDA graph.  Graphs are kept, keyed by the exact records (kernels, shapes
// and argument bytes), so a wave that recurs is replayed without rebuilding.
class WaveRunner {
  public:
    struct Stats {
        int64_t waves = 0, nodes = 0, records = 0, hits = 0, misses = 0;
    };
    WaveRunner() = default;
    WaveRunner(const WaveRunner &) = delete;
    WaveRunner &operator=(const WaveRunner &) = delete;
    ~WaveRunner() { clear(); }
    // merge and launch the records of recs[0 .. n) (one recorder per problem) on s
    cudaError_t run(Recorder *const *recs, int n, cudaStream_t s);
    void clear();
    Stats stats;

  private:
    struct Entry {
        std::vector<unsigned char> key;
        cudaGraphExec_t exec = nullptr;
        int64_t nodes = 0, records = 0;
    };
    std::vector<std::vector<Entry>> buckets_ = std::vector<std::vector<Entry>>(1024);
    size_t key_bytes_ = 0;
    std::vector<unsigned char> key_;
    cudaError_t build(Recorder *const *recs, int n, Entry &out);
};

// per-category kernel accounting (see hdg_profile_enable)
struct Prof {
    bool on = false;
    // cold-cache timing (hdg_profile_enable(h, 2)): a buffer of three times
    // the L2 size read before every bracketed launch
    void *evict_buf = nullptr;
    size_t evict_bytes = 0;
    uint32_t *evict_sink = nullptr;
    double ms[HDG_PROF_N] = {};
    int64_t launches[HDG_PROF_N] = {};
    struct Pending { int cat; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
};

}  // namespace hdg

// The handle (opaque to callers).
struct hdg_handle {
    std::string err;
    hdg_params prm{};
    int p = 0, pp = 0, np = 0, nK = 0, m = 0;
    int pf = 0;          // the facet-row kernels' block degree: trace dofs per facet pp = pf + 1
                         // (upwind: pp = p + 1; Lax-Friedrichs: pp = 2(p + 1))
    int N = 0, NF = 0, NT = 0, nv = 0, dim = 0;
    double tau_s = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool condensed = false;
    hdg::HostMesh hm;

    // device mesh / geometry
    double *d_ref = nullptr;        // packed reference matrices
    double *d_X = nullptr;          // [N][3][2]
    double *d_fcell = nullptr;      // [N][3] Coriolis at the cell vertices
    int32_t *d_facet_of = nullptr, *d_flip = nullptr;   // [N][3]
    int32_t *d_facet_cell = nullptr, *d_facet_edge = nullptr;  // [NF][2]
    int32_t *d_facet_verts = nullptr;  // [NF][2]
    int32_t *d_v2f_ptr = nullptr, *d_v2f = nullptr;
    int32_t *d_nbr = nullptr;       // [4][NF] neighbour facets of the facet-row operator

    // cell operators (component-major [j][N] layouts)
    double *d_Xb = nullptr;         // A^-1 B        [nK*m][N]
    double *d_Rm = nullptr;         // A^-1 Mass     [nK*nK][N]
    double *d_W = nullptr;          // C A^-1 Mass   [m*nK][N]
    // mixed modes: the same three matrices and the FP64 trace operator as
    // (hi, lo) float pairs for the two-float FP64 steps (k_ff.cu)
    float2 *d_Xb2 = nullptr, *d_Rm2 = nullptr, *d_W2 = nullptr, *d_Sval2 = nullptr;
    // C_K from geometry (two-float handles): pairs of H t_y, -H t_x, tau_s |e| per
    // cell and edge [N][3][3]; per row of C_K the cell nodes and pairs of the
    // nonzero reference facet entries [3(p+1)][p+1]; cz_ok once they are built
    float2 *d_cgeo = nullptr, *d_ctab_v = nullptr;
    int32_t *d_ctab_b = nullptr;
    bool cz_ok = false;
    double *d_Scell = nullptr;      // S_K           [N][m][m]
    // facet-row trace operator
    double *d_Sval = nullptr;       // 5(p+1)^2 values per facet, packed in 16-byte groups
    double *d_Dinv = nullptr;       // (p+1)^2 values per facet, packed likewise
    float *d_Sval32 = nullptr, *d_Dinv32 = nullptr;
    __nv_bfloat16 *d_Sval16 = nullptr;   // preconditioner copy (HDG_MIXED_BF16)
    int32_t *d_status = nullptr;    // device error flags: 1 zero pivot in A_K, 2 singular facet block,
                                    // 4 singular coarsest P1 operator, 8 coarse-cycle staging wait ran
                                    // out, 16 learned-sweep MMA wait ran out
    int device = -1;                // CUDA device current at hdg_setup
    double *noalloc_scratch = nullptr;   // device address of the fixed scratch array (noalloc.cu)

    std::vector<hdg::DevLevel> lev;
    int tail_start[2] = {0, 0};       // first P1 level of the single-CTA tail kernel (FP64, FP32)
    bool p1_fused = true;             // patch-fused P1 smoothing kernels on the levels above the tail
    int bs_facet = 256;               // threads per block of the facet-row kernels (autotuned)
    double *d_coarse_inv = nullptr;   // dense inverse of the coarsest P1 operator
    hdg::TailImage tail_img[2];       // shared-memory images of the tail levels (FP64, FP32)
    double *d_coarse_work = nullptr;
    double *d_coarse_fac = nullptr;   // row factors of one elimination step (coarsest levels above 256 vertices)
    hdg::Workspace *ws = nullptr;
    hdg::Prof prof;
    hdg::Learned lc;
    hdg::Imex imex;
    hdg::GalerkinDev gal;
    hdg::Rt0Dev rt0;
    // Lax-Friedrichs coarse solve: Chebyshev ellipse of D_c^-1 S_c, its Ritz values, step coefficients
    double cheb_c_theta = 0.0, cheb_c_delta2 = 0.0;
    std::vector<std::complex<double>> cheb_c_ritz;
    std::vector<double> cheb_c_omega, cheb_c_beta;
    bool has_f = false;               // a non-zero Coriolis field was given to hdg_setup
    // Chebyshev smoother (smoother 1): the ellipse, the Ritz values it was
    // fitted to, and per step k the sweep coefficients omega_k (of D^-1 r)
    // and beta_k (of x_k - x_{k-1})
    double cheb_theta = 0.0, cheb_delta2 = 0.0;
    std::vector<std::complex<double>> cheb_ritz;
    std::vector<double> cheb_omega, cheb_beta;
};

// ---------------------------------------------------------------- error helpers
#define HDG_CUDA_TRY(h, call)                                                        \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            (h)->err = std::string(#call) + ": " + cudaGetErrorString(e_);           \
            return HDG_ECUDA;                                                        \
        }                                                                            \
    } while (0)

namespace hdg {

// ---------------------------------------------------------------- kernel launchers
// condense / assembly (k_condense.cu)
// What a precision mode uses: two-float FP64 steps around FP32 inner FGMRES
// solves (HDG_MIXED_FP32 / _BF16); an FP64 Krylov space (HDG_FP64 and
// HDG_MIXED_FGMRES64); an FP32 preconditioner under the FP64 FGMRES
// (HDG_MIXED_FGMRES64).
inline bool mode_ff(const hdg_params &p) { return p.precision == HDG_MIXED_FP32 || p.precision == HDG_MIXED_BF16; }
inline bool mode_krylov64(const hdg_params &p) { return p.precision == HDG_FP64 || p.precision == HDG_MIXED_FGMRES64; }
inline bool mode_pre32(const hdg_params &p) { return p.precision == HDG_MIXED_FGMRES64; }

// dispatch a launch on the polynomial degree p (1..4) as a compile-time P
#define HDG_DISPATCH_P(p, CALL) \
    switch (p) {                \
        case 1: { constexpr int P = 1; CALL; } break; \
        case 2: { constexpr int P = 2; CALL; } break; \
        case 3: { constexpr int P = 3; CALL; } break; \
        case 4: { constexpr int P = 4; CALL; } break; \
        default: return cudaErrorInvalidValue;        \
    }

// Spectral estimate for the Chebyshev smoother (spectrum.cpp, host): the
// eigenvalues of an n x n upper Hessenberg matrix (row-major), and the
// ellipse (centre theta, squared focal half-distance delta2) fitted to Ritz
// values with real extent [lower b, b], b = grow * max Re.
std::vector<std::complex<double>> hessenberg_eigenvalues(const std::vector<double> &H, int n);
void chebyshev_ellipse(const std::vector<std::complex<double>> &ritz, double lower, double grow, double &theta,
                       double &delta2);

// Kernel accounting for entry points defined outside api.cu: counts nk
// launches in category cat and, with timing on, brackets what fn enqueues
// with events on the handle's stream (see hdg_profile_enable).
cudaError_t account_launch(hdg_handle *h, int cat, int nk, const std::function<cudaError_t()> &fn);
// Look up the device address of the no-allocation scratch array on the
// current device and keep it in the handle (noalloc.cu; called by hdg_setup).
cudaError_t noalloc_prepare(hdg_handle *h);

// read a buffer larger than L2 so that the next kernel's data comes from DRAM (k_measure.cu)
cudaError_t launch_l2_evict(const void *buf, size_t bytes, uint32_t *sink, cudaStream_t s);

// IMEX rates (k_imex.cu): upwind trace of the state, then M^-1 N(q) (nu, nh;
// skipped when null) and M^-1 L(q) (lu, lh) per cell
cudaError_t launch_imex_rates(hdg_handle *h, const double *u, const double *hh, double *nu, double *nh, double *lu,
                              double *lh);
void imex_release(hdg_handle *h);

// dispatch a facet-row kernel on the degree of its trace blocks (h->pf: the
// blocks are (pf+1) x (pf+1)); pf = 5 (the vector trace at p = 2) exists in FP64 only
#define HDG_DISPATCH_PF(pf, T, CALL) \
    switch (pf) {                    \
        case 1: { constexpr int P = 1; CALL; } break; \
        case 2: { constexpr int P = 2; CALL; } break; \
        case 3: { constexpr int P = 3; CALL; } break; \
        case 4: { constexpr int P = 4; CALL; } break; \
        case 5: if constexpr (std::is_same<T, double>::value) { constexpr int P = 5; CALL; } \
                else { return cudaErrorInvalidValue; } break;                             \
        default: return cudaErrorInvalidValue;        \
    }

// Lax-Friedrichs variant (k_lf.cu)
cudaError_t launch_condense_lf(hdg_handle *h);
cudaError_t launch_rhs_lf(hdg_handle *h, const double *r_u, const double *r_h, double *g, double *ycell);
cudaError_t launch_recover_lf(hdg_handle *h, const double *r_u, const double *r_h, const double *lam, double *u,
                              double *hout);
cudaError_t launch_rt0_assemble(hdg_handle *h);
cudaError_t launch_rt0_apply_dinv(hdg_handle *h, const double *x, double *y);
cudaError_t launch_rt0_cheb(hdg_handle *h, const double *r, const double *x, const double *xprev, double *out,
                            double omega, double beta);
cudaError_t launch_rt0_restrict(hdg_handle *h, const double *r, double *rc);
cudaError_t launch_rt0_prolong_add(hdg_handle *h, const double *ec, double *x);

cudaError_t launch_condense(hdg_handle *h);
cudaError_t launch_assemble(hdg_handle *h);
cudaError_t launch_p1_assemble(hdg_handle *h, DevLevel &L, double tau, double gH, int rotating);
// every P1 level operator as the Galerkin product of the trace operator (k_galerkin.cu)
cudaError_t launch_p1_galerkin(hdg_handle *h);
cudaError_t launch_dense_inverse(hdg_handle *h, const DevLevel &L, double *work, double *inv, int n);
// true when launch_condense writes the mixed handles' float-pair matrices
// (X_B, R_M, W_K) itself, so that no FP64 copy of them exists to split
bool condense_writes_pairs(const hdg_handle *h);
// a tail level's ELL arrays in the staged layout: values (tsz bytes each)
// slot-major into A_dst, columns as 16-bit indices into col_dst
cudaError_t launch_tail_pack(const int32_t *col, const void *A, size_t tsz, int nv, int W, void *col_dst, void *A_dst,
                             cudaStream_t s);
cudaError_t launch_to_f32(const double *x, float *y, size_t n, cudaStream_t s);

// trace-space kernels (k_trace.cu); vectors in the internal layout [pp][NF]
cudaError_t launch_to_internal(hdg_handle *h, const double *ext, double *in);
cudaError_t launch_repack(hdg_handle *h);
// index of element j of facet e in an operator array packed in groups of G
inline __host__ __device__ size_t packed_index(size_t j, size_t e, size_t NF, size_t G) {
    return ((j / G) * NF + e) * G + j % G;
}
cudaError_t launch_to_external(hdg_handle *h, const double *in, double *ext);
// optional hand-over of ||v||^2 by the kernel that forms v: block partials,
// the reduction counter, the device result and, with pub non-null, the
// page-locked word the host polls (sequence number seq)
// The start of an FP32 inner solve, written by the kernel that forms its
// right-hand side v in FP64 (b32 null: not wanted): b32 = fp32(v * scale),
// z32 = 0 (the zero initial guess) and, by the block that completes the norm,
// root_a = root_b = ||v|| * scale (scale a power of two, so exact).
struct F32Copy {
    float *b32 = nullptr;
    float *z32 = nullptr;
    double scale = 1.0;
    double *root_a = nullptr;
    double *root_b = nullptr;
};
struct NormOut {
    double *partial = nullptr;
    unsigned int *counter = nullptr;
    double *out = nullptr;
    HostValue *pub = nullptr;
    int32_t seq = 0;
    F32Copy f32 = F32Copy();
};
cudaError_t launch_rhs(hdg_handle *h, const double *r_u, const double *r_h, double *g, double *ycell,
                       const NormOut &nrm = NormOut());
cudaError_t launch_rhs_gather(hdg_handle *h, const double *ycell, double *g, const NormOut &nrm = NormOut());
// two-float versions of the FP64 steps (mixed modes, k_ff.cu)
cudaError_t launch_split(const double *a, float2 *out, size_t n, cudaStream_t s);
// a per-cell matrix [rows][cols][N] split into pairs of row entries, tiled by 32 cells:
// [ceil(N/32)][rows][(cols+1)/2][32] (float4)
cudaError_t launch_split_pairs(const double *a, float2 *out, int rows, int cols, size_t N, cudaStream_t s);
// facets per block of the two-float residual (its grid: ceil(NF / kResFFFacets)
// blocks, each writing one partial sum)
constexpr int kResFFFacets = 64;
// x2 += scale[0] * d in two-float arithmetic (first: x2 = scale[0] * d)
cudaError_t launch_ff_axpy(float2 *x2, const float *d, const double *scale, size_t n, bool first, cudaStream_t s);
// the last cycle of a mixed inner solve: y = R^-1 s (k x k rotated Hessenberg
// triangle), d = x + Z y (x null: zero), x2 += scale[0] * d in two-float
// arithmetic (first: x2 = scale[0] * d); k <= 64
cudaError_t launch_ff_finish(const double *Hm, int ldh, const double *sv, int k, const float *Z, size_t ld,
                             const float *x, float2 *x2, const double *scale, size_t n, bool first, cudaStream_t s);
// a = b = hi + lo of each pair (b may be null)
cudaError_t launch_ff_join(const float2 *x2, double *a, double *b, size_t n, cudaStream_t s);
cudaError_t launch_residual_ff(hdg_handle *h, const double *b, const float2 *x2, double *res,
                               double *partial = nullptr, unsigned int *counter = nullptr, double *out = nullptr,
                               HostValue *pub = nullptr, int32_t seq = 0, const F32Copy &c32 = F32Copy());
// (r_u, r_h may be device aliases of page-locked host memory; copy_u / copy_h,
// if non-null, receive a device copy of them)
cudaError_t launch_rhs_ff(hdg_handle *h, const double *r_u, const double *r_h, double *g, double *ycell,
                          double *copy_u, double *copy_h, const NormOut &nrm = NormOut());
cudaError_t launch_recover_ff(hdg_handle *h, const double *r_u, const double *r_h, const double *lam, double *u,
                              double *hout);
// step 1 of a solve keeping z_K = R_M r_K (pairs, [nK][N]) for step 3, C_K z_K
// formed from the cell geometry (handles with cz_ok); step 3 from that z
cudaError_t launch_rhs_z(hdg_handle *h, const double *r_u, const double *r_h, double *g, double *ycell, float2 *z2,
                         double *copy_u, double *copy_h, const NormOut &nrm = NormOut());
cudaError_t launch_recover_z(hdg_handle *h, const float2 *z2, const double *lam, double *u, double *hout);
// whether the last solve's step 1 kept z_K (hdg_recover_dev may then take NULL right-hand sides)
bool solve_kept_z(const hdg_handle *h);
cudaError_t launch_recover(hdg_handle *h, const double *r_u, const double *r_h, const double *lam,
                           double *u, double *hout);

// P1 multigrid kernels (k_p1.cu)
template <typename T>
cudaError_t launch_p1_jacobi(const DevLevel &L, const T *A, const T *dinv, const T *b, const T *x,
                             T *xout, T omega, bool first, cudaStream_t s);
template <typename T>
cudaError_t launch_p1_prolong_add(const DevLevel &coarse, int nv_fine, const T *ec, T *xf, cudaStream_t s);
template <typename T>
cudaError_t launch_p1_down(const DevLevel &fine, const DevLevel &coarse, const T *A_f, const T *b_f, const T *x_f,
                           const T *dinv_c, T omega, T *b_c, T *x_c, cudaStream_t s);
template <typename T>
cudaError_t launch_p1_up(const DevLevel &fine, const DevLevel &coarse, const T *A_f, const T *dinv_f, const T *b_f,
                         const T *x_f, const T *ec, T *xout, T omega, cudaStream_t s);
// one launch per patch: the last pre-smoothing sweep, the residual and the
// restriction (down); the prolongation with both post-smoothing sweeps (up)
template <typename T>
bool p1_patch_ok(const DevLevel &L);   // the level's patches suit these kernels in precision T
template <typename T>
cudaError_t launch_p1_down_fused(const DevLevel &fine, const DevLevel &coarse, const T *A_f, const T *dinv_f,
                                 const T *b_f, const T *x_f, T *xout_f, const T *dinv_c, T omega, T *b_c, T *x_c,
                                 cudaStream_t s);
template <typename T>
cudaError_t launch_p1_up_fused(const DevLevel &fine, const DevLevel &coarse, const T *A_f, const T *dinv_f,
                               const T *b_f, const T *x_f, const T *ec, T *xout, T omega, cudaStream_t s);
template <typename T>
cudaError_t launch_p1_tail(const TailArgs &a, size_t smem, cudaStream_t s);
// x = inv b on the coarsest level (n vertices, FP64 inverse) over many CTAs
template <typename T>
cudaError_t launch_p1_coarse_dense(const double *inv, int n, const T *b, T *x, cudaStream_t s);
// coarsest levels above this size alone in the tail take the multi-CTA product
constexpr int kTailDenseMax = 256;

// Krylov kernels (k_krylov.cu)
template <typename T>
cudaError_t launch_multidot(const T *V, size_t ld, int k, const T *w, size_t n, double *partial,
                            int nchunk, cudaStream_t s);
// v . w in one launch (partials per chunk, then the last block adds them; the
// same order and result as multidot + reduce_partials with k = 1)
template <typename T>
cudaError_t launch_dot1(const T *v, const T *w, size_t n, double *partial, int nchunk, unsigned int *counter,
                        double *out, HostValue *pub, int32_t seq, double *root_a, double *root_b, cudaStream_t s);
cudaError_t launch_reduce_partials(const double *partial, int k, int nchunk, double *out, cudaStream_t s,
                                   HostValue *pub = nullptr, int32_t seq = 0, double *root_a = nullptr,
                                   double *root_b = nullptr);
template <typename T>
cudaError_t launch_multi_axpy(T *w, const T *V, size_t ld, int k, const double *coef, double sign,
                              size_t n, cudaStream_t s);
template <typename T>
cudaError_t launch_scale_copy(const T *w, T *v, const double *denom, size_t n, cudaStream_t s);
cudaError_t launch_hessenberg_solve(const double *Hm, int ldh, const double *sv, int k, double *y,
                                    cudaStream_t s);
template <typename T>
cudaError_t launch_fill(T *x, T v, size_t n, cudaStream_t s);
template <typename T>
cudaError_t launch_gs_step(const T *V, size_t ld, int j, T *w, double *partial, unsigned int *counter, int nblk,
                           double *h1, double *h2, double *nrm2, double *Hm, int ldh, double *cs, double *sn,
                           double *sv, const double *bnorm, ReadBack *rb, ReadBack *host_rb, T *vnext, bool reorth, bool scale,
                           cudaStream_t s);
int learned_n_params(int p, int hid);
cudaError_t launch_learned_infer(hdg_handle *h, const float *r, const float *x, float *xout);
cudaError_t launch_learned_infer_tc(hdg_handle *h, const float *r, const float *x, float *xout);
cudaError_t launch_learned_tc_weights(hdg_handle *h);
size_t learned_tc_image_elems(int p, int hid);
cudaError_t launch_learned_forward(hdg_handle *h, const float *r, float *c);
cudaError_t launch_learned_applyT(hdg_handle *h, const float *x, float *y);
cudaError_t launch_learned_backward(hdg_handle *h, const float *gc, const double *coef);
cudaError_t launch_adam(hdg_handle *h, float lr, int t);
cudaError_t launch_normalize32(const float *src, float *dst, const double *nrm2, size_t n, cudaStream_t s);
cudaError_t launch_to_internal32(hdg_handle *h, const float *ext, float *in);
cudaError_t launch_to_external32(hdg_handle *h, const float *in, float *ext);
cudaError_t launch_scale_round(const double *w, const double *hnext, double *v64, float *v32, size_t n,
                               cudaStream_t s);
cudaError_t launch_widen(const float *a, double *b, size_t n, cudaStream_t s);
cudaError_t launch_d2f_scaled(const double *x, float *y, const double *scale, size_t n, cudaStream_t s);
// y = float(x / scale[0]), z = 0 and ||y||^2 into out[0] (its root into root_a /
// root_b), nchunk blocks, deterministic
cudaError_t launch_d2f_norm(const double *x, float *y, float *z, const double *scale, size_t n, double *partial,
                            int nchunk, unsigned int *counter, double *out, double *root_a, double *root_b,
                            cudaStream_t s);

}  // namespace hdg
