// Galerkin coarse operators for the P1 levels (coarse_mode = 2): the
// alternative of the footnote in Sec. 4.4, A_0 = pi^T S pi on the fine P1
// level (pi the injection of P1 into the trace space, S the trace operator)
// and A_{l+1} = P_l^T A_l P_l on the nested coarser levels (P_l linear
// interpolation).  Both keep the P1 stencil (vertices sharing a cell), so the
// level operators reuse the padded ELL structure of the rediscretised ones.
//
// Every ELL slot sums a list of contributions built on the host at set-up,
// in a fixed order:
//   level 0: for facet e, block b of its facet row (b = 0: e itself,
//            b = 1 + 2s + k: facet (i_s + 1 + k) % 3 of its cell s), and the
//            ends sv, sw of e and of the block's facet, the slot of
//            (vertex sv of e, vertex sw of the block's facet) receives
//            sum_{r,c} W(sv, r) S_{e,b}[r][c] W(sw, c),  W(0, t) = 1 - t/p,
//            W(1, t) = t/p (the nodal weights of pi along a facet);
//   level l+1: the slot (I, J) receives w_iI w_jJ A_l[i, j] for every slot
//            (i, j) of level l and every parent I of i, J of j (weight 1 for
//            a coincident vertex, 1/2 for a midpoint).
#include "common.h"

#include <algorithm>

namespace hdg {

namespace {

// slot of column c in row v of a padded ELL level (the first match: the
// diagonal for c = v, since unused slots repeat v after it), -1 if absent
int ell_slot(const HostLevel &L, int v, int c) {
    for (int q = 0; q < L.width; ++q)
        if (L.col[size_t(v) * L.width + q] == c) return v * L.width + q;
    return -1;
}

}  // namespace

std::string build_galerkin_lists(const HostMesh &hm, GalerkinHost &g) {
    g = GalerkinHost();
    const HostLevel &L0 = hm.levels[0];
    const int NF = hm.nf;
    // facet-row neighbours exactly as the facet-row assembly orders them
    std::vector<std::vector<int32_t>> slot_codes(size_t(L0.nv) * L0.width);
    for (int e = 0; e < NF; ++e) {
        int nb[5];
        nb[0] = e;
        for (int s = 0; s < 2; ++s) {
            const int K = hm.facet_cell[2 * e + s], I = hm.facet_edge[2 * e + s];
            for (int k = 0; k < 2; ++k) nb[1 + 2 * s + k] = hm.facet_of[3 * K + (I + 1 + k) % 3];
        }
        for (int b = 0; b < 5; ++b)
            for (int sv = 0; sv < 2; ++sv)
                for (int sw = 0; sw < 2; ++sw) {
                    const int v = hm.facet_verts[2 * e + sv], w = hm.facet_verts[2 * nb[b] + sw];
                    const int q = ell_slot(L0, v, w);
                    if (q < 0) return "Galerkin coarse operator: a facet coupling outside the P1 stencil";
                    slot_codes[size_t(q)].push_back(e * 20 + b * 4 + sv * 2 + sw);
                }
    }
    g.ptr0.assign(slot_codes.size() + 1, 0);
    for (size_t q = 0; q < slot_codes.size(); ++q) {
        g.ptr0[q + 1] = g.ptr0[q] + int32_t(slot_codes[q].size());
        g.code0.insert(g.code0.end(), slot_codes[q].begin(), slot_codes[q].end());
    }
    // coarser levels
    for (size_t l = 0; l + 1 < hm.levels.size(); ++l) {
        const HostLevel &F = hm.levels[l], &Cl = hm.levels[l + 1];
        std::vector<std::vector<std::pair<int32_t, double>>> lists(size_t(Cl.nv) * Cl.width);
        auto parents = [&](int i, int *par, double *w) {
            const int a = Cl.parent[2 * size_t(i)], b = Cl.parent[2 * size_t(i) + 1];
            if (a == b) {
                par[0] = a; w[0] = 1.0;
                return 1;
            }
            par[0] = a; w[0] = 0.5;
            par[1] = b; w[1] = 0.5;
            return 2;
        };
        for (int i = 0; i < F.nv; ++i) {
            int pi[2], pj[2];
            double wi[2], wj[2];
            const int ni = parents(i, pi, wi);
            for (int s = 0; s < F.width; ++s) {
                const int q = i * F.width + s, j = F.col[size_t(q)];
                if (j == i && q != F.diag[size_t(i)]) continue;      // unused slot
                const int nj = parents(j, pj, wj);
                for (int a = 0; a < ni; ++a)
                    for (int b = 0; b < nj; ++b) {
                        const int Q = ell_slot(Cl, pi[a], pj[b]);
                        if (Q < 0) return "Galerkin coarse operator: a coupling outside the coarse P1 stencil";
                        lists[size_t(Q)].push_back({q, wi[a] * wj[b]});
                    }
            }
        }
        std::vector<int32_t> ptr(lists.size() + 1, 0), idx;
        std::vector<double> w;
        for (size_t Q = 0; Q < lists.size(); ++Q) {
            ptr[Q + 1] = ptr[Q] + int32_t(lists[Q].size());
            for (auto &pr : lists[Q]) {
                idx.push_back(pr.first);
                w.push_back(pr.second);
            }
        }
        g.ptr.push_back(std::move(ptr));
        g.idx.push_back(std::move(idx));
        g.w.push_back(std::move(w));
    }
    return "";
}

namespace {

template <int P>
__global__ void galerkin0_kernel(int nnz, int NF, const int32_t *__restrict__ ptr, const int32_t *__restrict__ code,
                                 const double *__restrict__ Sval, double *__restrict__ A) {
    constexpr int PP = P + 1;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nnz) return;
    double acc = 0.0;
    for (int k = ptr[q]; k < ptr[q + 1]; ++k) {
        const int c0 = code[k], e = c0 / 20, rem = c0 % 20, b = rem / 4, sv = (rem / 2) % 2, sw = rem % 2;
        double blk = 0.0;
#pragma unroll
        for (int r = 0; r < PP; ++r) {
            const double wr = sv ? double(r) / P : 1.0 - double(r) / P;
            double row = 0.0;
#pragma unroll
            for (int c = 0; c < PP; ++c) {
                const double wc = sw ? double(c) / P : 1.0 - double(c) / P;
                row = fma(Sval[packed_index(size_t((r * 5 + b) * PP + c), size_t(e), size_t(NF), 2)], wc, row);
            }
            blk = fma(wr, row, blk);
        }
        acc += blk;
    }
    A[q] = acc;
}

__global__ void galerkin_coarse_kernel(int nnz, const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                                       const double *__restrict__ w, const double *__restrict__ Af,
                                       double *__restrict__ Ac) {
    const int Q = blockIdx.x * blockDim.x + threadIdx.x;
    if (Q >= nnz) return;
    double acc = 0.0;
    for (int k = ptr[Q]; k < ptr[Q + 1]; ++k) acc = fma(w[k], Af[idx[k]], acc);
    Ac[Q] = acc;
}

__global__ void galerkin_dinv_kernel(int nv, const int32_t *__restrict__ diag, const double *__restrict__ A,
                                     double *__restrict__ dinv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nv) dinv[i] = 1.0 / A[diag[i]];
}

}  // namespace

cudaError_t launch_p1_galerkin(hdg_handle *h) {
    const GalerkinDev &G = h->gal;
    DevLevel &L0 = h->lev[0];
    HDG_DISPATCH_P(h->p, (galerkin0_kernel<P><<<(L0.nnz + 255) / 256, 256, 0, h->stream>>>(
                             L0.nnz, h->NF, G.ptr0, G.code0, h->d_Sval, L0.A)));
    cudaError_t e = cudaGetLastError();
    for (size_t l = 0; l + 1 < h->lev.size() && e == cudaSuccess; ++l) {
        DevLevel &C = h->lev[l + 1];
        galerkin_coarse_kernel<<<(C.nnz + 255) / 256, 256, 0, h->stream>>>(C.nnz, G.ptr[l], G.idx[l], G.w[l],
                                                                           h->lev[l].A, C.A);
        e = cudaGetLastError();
    }
    for (auto &L : h->lev) {
        if (e != cudaSuccess) break;
        galerkin_dinv_kernel<<<(L.nv + 255) / 256, 256, 0, h->stream>>>(L.nv, L.diag, L.A, L.dinv);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace hdg
