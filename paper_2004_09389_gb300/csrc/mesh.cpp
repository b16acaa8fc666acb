// Host-side mesh processing at hdg_setup: validation, facet numbering and
// orientation, local 2-D cell coordinates, vertex->facet incidence for the
// P1 restriction, and the nested P1 levels with their geometric mass and
// stiffness matrices (Sec. 4.4: the upwind coarse space is P1 on the same
// triangulation; coarser P1 levels serve the geometric V-cycle).
#include "common.h"

#include <algorithm>
#include <cmath>
#include <unordered_map>

namespace hdg {

namespace {

std::string local_coords(const hdg_mesh_level &L, std::vector<double> &X) {
    X.assign(size_t(L.n_cells) * 6, 0.0);
    for (int K = 0; K < L.n_cells; ++K) {
        double P[3][3] = {};
        for (int i = 0; i < 3; ++i) {
            int v = L.cell_vertices[3 * K + i];
            for (int d = 0; d < L.dim; ++d) P[i][d] = L.vertex_xyz[size_t(v) * L.dim + d];
            if (L.dim == 2 && L.cell_shift) {
                P[i][0] += L.cell_shift[(size_t(K) * 3 + i) * 2 + 0];
                P[i][1] += L.cell_shift[(size_t(K) * 3 + i) * 2 + 1];
            }
        }
        double *x = &X[size_t(K) * 6];
        if (L.dim == 2) {
            for (int i = 0; i < 3; ++i) { x[2 * i] = P[i][0]; x[2 * i + 1] = P[i][1]; }
        } else {
            double d1[3], d2[3], e1[3], nn[3], e2[3];
            for (int d = 0; d < 3; ++d) { d1[d] = P[1][d] - P[0][d]; d2[d] = P[2][d] - P[0][d]; }
            double l1 = std::sqrt(d1[0] * d1[0] + d1[1] * d1[1] + d1[2] * d1[2]);
            if (!(l1 > 0)) return "degenerate cell";
            for (int d = 0; d < 3; ++d) e1[d] = d1[d] / l1;
            nn[0] = d1[1] * d2[2] - d1[2] * d2[1];
            nn[1] = d1[2] * d2[0] - d1[0] * d2[2];
            nn[2] = d1[0] * d2[1] - d1[1] * d2[0];
            double ln = std::sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
            if (!(ln > 0)) return "degenerate cell";
            for (int d = 0; d < 3; ++d) nn[d] /= ln;
            e2[0] = nn[1] * e1[2] - nn[2] * e1[1];
            e2[1] = nn[2] * e1[0] - nn[0] * e1[2];
            e2[2] = nn[0] * e1[1] - nn[1] * e1[0];
            for (int i = 0; i < 3; ++i) {
                double dd[3] = {P[i][0] - P[0][0], P[i][1] - P[0][1], P[i][2] - P[0][2]};
                x[2 * i] = dd[0] * e1[0] + dd[1] * e1[1] + dd[2] * e1[2];
                x[2 * i + 1] = dd[0] * e2[0] + dd[1] * e2[1] + dd[2] * e2[2];
            }
        }
        double det = (x[2] - x[0]) * (x[5] - x[1]) - (x[4] - x[0]) * (x[3] - x[1]);
        if (!(det > 0)) return "cell " + std::to_string(K) + " is not counter-clockwise";
    }
    return "";
}

std::string check_level(const hdg_mesh_level &L, const char *what) {
    if (L.n_vertices <= 0 || L.n_cells <= 0) return std::string(what) + ": empty mesh";
    if (L.dim != 2 && L.dim != 3) return std::string(what) + ": dim must be 2 or 3";
    if (!L.vertex_xyz || !L.cell_vertices) return std::string(what) + ": NULL array";
    for (long i = 0; i < 3L * L.n_cells; ++i)
        if (L.cell_vertices[i] < 0 || L.cell_vertices[i] >= L.n_vertices)
            return std::string(what) + ": vertex index out of range";
    return "";
}

// P1 element data on one level and the structure of the level operator:
// per cell the 3x3 mass, stiffness (grad L_b, grad L_a) and skew
// (J grad L_b, grad L_a) matrices (J the rotation by 90 degrees in the cell's
// plane).  The operator is stored in a padded row-major ELL layout: width W =
// the longest row rounded up to a multiple of 4 (rows start on 16-byte
// boundaries and load as 16-byte vectors); slot q of row v sits at v * W + q;
// row v lists its columns in increasing order in slots 0..len-1 and points the
// remaining slots at v itself with no contributions (value 0).  Every slot has
// the list of (cell, a, b) that contribute to it, in cell order, so the device
// sums each entry in a fixed order.
void p1_matrices(HostLevel &hl) {
    hl.elem.assign(size_t(hl.nc) * 27, 0.0);
    std::vector<std::vector<std::pair<int, int>>> rows(hl.nv);   // (column, contribution code)
    for (int K = 0; K < hl.nc; ++K) {
        const double *x = &hl.X[size_t(K) * 6];
        double J00 = x[2] - x[0], J01 = x[4] - x[0], J10 = x[3] - x[1], J11 = x[5] - x[1];
        double det = J00 * J11 - J01 * J10;
        // gradients of the barycentric coordinates: grad L = J^-T grad_ref L
        double gref[3][2] = {{-1, -1}, {1, 0}, {0, 1}};
        double G[3][2];
        for (int a = 0; a < 3; ++a) {
            G[a][0] = (J11 * gref[a][0] - J10 * gref[a][1]) / det;
            G[a][1] = (-J01 * gref[a][0] + J00 * gref[a][1]) / det;
        }
        double *el = &hl.elem[size_t(K) * 27];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                const int ab = a * 3 + b;
                el[ab] = det / 24.0 * (a == b ? 2.0 : 1.0);
                el[9 + ab] = 0.5 * det * (G[a][0] * G[b][0] + G[a][1] * G[b][1]);
                // (J g_b) . g_a with J g = (-g_y, g_x)
                el[18 + ab] = 0.5 * det * (G[a][0] * (-G[b][1]) + G[a][1] * G[b][0]);
                rows[hl.cells[3 * K + a]].push_back({hl.cells[3 * K + b], K * 9 + ab});
            }
    }
    // merge equal columns: per row the distinct columns and their contribution ranges
    std::vector<std::vector<int>> cols(hl.nv);
    std::vector<std::vector<std::vector<int>>> codes(hl.nv);
    int W = 1;
    for (int v = 0; v < hl.nv; ++v) {
        auto &r = rows[v];
        std::stable_sort(r.begin(), r.end(), [](auto &a, auto &b) { return a.first < b.first; });
        for (size_t k = 0; k < r.size();) {
            size_t k2 = k;
            cols[v].push_back(r[k].first);
            codes[v].emplace_back();
            while (k2 < r.size() && r[k2].first == r[k].first) codes[v].back().push_back(r[k2++].second);
            k = k2;
        }
        W = std::max(W, int(cols[v].size()));
    }
    W = (W + 3) / 4 * 4;
    hl.width = W;
    hl.col.assign(size_t(W) * hl.nv, 0);
    hl.diag.assign(hl.nv, -1);
    hl.contrib_ptr.assign(1, 0);
    hl.contrib.clear();
    for (int v = 0; v < hl.nv; ++v)
        for (int q = 0; q < W; ++q) {
            const size_t slot = size_t(v) * W + q;
            if (q < int(cols[v].size())) {
                hl.col[slot] = cols[v][q];
                if (cols[v][q] == v) hl.diag[v] = int(slot);
                for (int c : codes[v][q]) hl.contrib.push_back(c);
            } else {
                hl.col[slot] = v;
            }
            hl.contrib_ptr.push_back(int(hl.contrib.size()));
        }
}

}  // namespace

std::string build_host_mesh(const hdg_mesh_desc *desc, HostMesh &hm) {
    if (!desc) return "mesh descriptor is NULL";
    const hdg_mesh_level &F = desc->fine;
    std::string e = check_level(F, "fine level");
    if (!e.empty()) return e;
    if (F.dim == 2 && !F.cell_shift) return "flat meshes need cell_shift (periodic unwrapping)";
    hm.dim = F.dim;
    hm.nv = F.n_vertices;
    hm.nc = F.n_cells;
    hm.cells.assign(F.cell_vertices, F.cell_vertices + 3 * size_t(F.n_cells));
    e = local_coords(F, hm.X);
    if (!e.empty()) return "fine level: " + e;

    // facets in order of first appearance over (cell, local edge)
    hm.facet_of.assign(3 * size_t(hm.nc), -1);
    hm.flip.assign(3 * size_t(hm.nc), 0);
    std::unordered_map<uint64_t, int> ids;
    ids.reserve(size_t(hm.nc) * 2);
    std::vector<int> count;
    hm.facet_verts.clear();
    hm.facet_cell.clear();
    hm.facet_edge.clear();
    for (int K = 0; K < hm.nc; ++K) {
        for (int i = 0; i < 3; ++i) {
            int a = hm.cells[3 * K + (i + 1) % 3], b = hm.cells[3 * K + (i + 2) % 3];
            if (a == b) return "cell with a repeated vertex";
            int lo = std::min(a, b), hi = std::max(a, b);
            uint64_t key = (uint64_t(uint32_t(lo)) << 32) | uint32_t(hi);
            auto it = ids.find(key);
            int f;
            if (it == ids.end()) {
                f = int(count.size());
                ids.emplace(key, f);
                count.push_back(0);
                hm.facet_verts.push_back(lo);
                hm.facet_verts.push_back(hi);
                hm.facet_cell.push_back(K);
                hm.facet_cell.push_back(-1);
                hm.facet_edge.push_back(i);
                hm.facet_edge.push_back(-1);
            } else {
                f = it->second;
                if (count[f] >= 2) return "a facet has more than two cells (non-manifold mesh)";
                hm.facet_cell[2 * f + 1] = K;
                hm.facet_edge[2 * f + 1] = i;
            }
            count[f] += 1;
            hm.facet_of[3 * K + i] = f;
            hm.flip[3 * K + i] = a > b ? 1 : 0;
        }
    }
    hm.nf = int(count.size());
    for (int f = 0; f < hm.nf; ++f)
        if (count[f] != 2) return "mesh is not closed: a facet has only one cell";
    // the two cells must traverse a shared facet in opposite directions
    for (int f = 0; f < hm.nf; ++f) {
        int K0 = hm.facet_cell[2 * f], K1 = hm.facet_cell[2 * f + 1];
        int i0 = hm.facet_edge[2 * f], i1 = hm.facet_edge[2 * f + 1];
        if (hm.flip[3 * K0 + i0] == hm.flip[3 * K1 + i1]) return "inconsistent cell orientation";
    }

    // vertex -> incident facet ends
    hm.v2f_ptr.assign(hm.nv + 1, 0);
    for (int f = 0; f < hm.nf; ++f) {
        hm.v2f_ptr[hm.facet_verts[2 * f] + 1]++;
        hm.v2f_ptr[hm.facet_verts[2 * f + 1] + 1]++;
    }
    for (int v = 0; v < hm.nv; ++v) hm.v2f_ptr[v + 1] += hm.v2f_ptr[v];
    hm.v2f.assign(hm.v2f_ptr[hm.nv], 0);
    {
        std::vector<int> fill(hm.v2f_ptr.begin(), hm.v2f_ptr.end() - 1);
        for (int f = 0; f < hm.nf; ++f) {
            hm.v2f[fill[hm.facet_verts[2 * f]]++] = 2 * f;
            hm.v2f[fill[hm.facet_verts[2 * f + 1]]++] = 2 * f + 1;
        }
    }

    // P1 levels
    hm.levels.clear();
    HostLevel L0;
    L0.nv = hm.nv;
    L0.nc = hm.nc;
    L0.X = hm.X;
    L0.cells = hm.cells;
    p1_matrices(L0);
    hm.levels.push_back(std::move(L0));
    if (desc->n_coarse < 0 || (desc->n_coarse > 0 && !desc->coarse)) return "bad coarse level list";
    for (int l = 0; l < desc->n_coarse; ++l) {
        const hdg_mesh_level &C = desc->coarse[l];
        std::string what = "coarse level " + std::to_string(l);
        e = check_level(C, what.c_str());
        if (!e.empty()) return e;
        if (C.dim != F.dim) return what + ": dim differs from the fine level";
        if (C.dim == 2 && !C.cell_shift) return what + ": flat meshes need cell_shift";
        if (!C.parent) return what + ": parent array is NULL";
        HostLevel hl;
        hl.nv = C.n_vertices;
        hl.nc = C.n_cells;
        hl.vdim = C.dim;
        hl.vxyz.assign(C.vertex_xyz, C.vertex_xyz + size_t(C.n_vertices) * C.dim);
        hl.cells.assign(C.cell_vertices, C.cell_vertices + 3 * size_t(C.n_cells));
        e = local_coords(C, hl.X);
        if (!e.empty()) return what + ": " + e;
        const int nvf = hm.levels.back().nv;
        hl.parent.assign(C.parent, C.parent + 2 * size_t(nvf));
        for (long i = 0; i < 2L * nvf; ++i)
            if (hl.parent[i] < 0 || hl.parent[i] >= hl.nv) return what + ": parent index out of range";
        // restriction (transpose of the midpoint prolongation)
        std::vector<std::vector<std::pair<int, double>>> ch(hl.nv);
        for (int i = 0; i < nvf; ++i) {
            int a = hl.parent[2 * i], b = hl.parent[2 * i + 1];
            if (a == b) ch[a].push_back({i, 1.0});
            else { ch[a].push_back({i, 0.5}); ch[b].push_back({i, 0.5}); }
        }
        hl.child_ptr.assign(hl.nv + 1, 0);
        for (int c = 0; c < hl.nv; ++c) {
            for (auto &pr : ch[c]) { hl.child_idx.push_back(pr.first); hl.child_w.push_back(pr.second); }
            hl.child_ptr[c + 1] = int(hl.child_idx.size());
        }
        p1_matrices(hl);
        hm.levels.push_back(std::move(hl));
    }
    if (hm.levels.back().nv > 1024)
        return "the coarsest P1 level has more than 1024 vertices; pass more coarse levels";
    // patches only where their per-row copies stay small (a few MB): on larger
    // levels the copies displace the facet operator from L2 and the unfused
    // kernels measured faster
    for (int l = 0; l + 1 < int(hm.levels.size()); ++l)
        if (hm.levels[l].nv <= kPatchMaxVertices) build_p1_patches(hm, l, 128);
    return "";
}

namespace {

// recursive coordinate bisection of ids[lo, hi) into parts of at most maxsz
// vertices: split at the median of the coordinate with the largest extent
// (ties by vertex id, so the result is deterministic)
void rcb(std::vector<int> &ids, int lo, int hi, const std::vector<double> &xyz, int dim, int maxsz,
         std::vector<int> &part, int &np) {
    if (hi - lo <= maxsz) {
        for (int i = lo; i < hi; ++i) part[ids[i]] = np;
        ++np;
        return;
    }
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
    for (int i = lo; i < hi; ++i)
        for (int d = 0; d < dim; ++d) {
            const double x = xyz[size_t(ids[i]) * dim + d];
            mn[d] = std::min(mn[d], x);
            mx[d] = std::max(mx[d], x);
        }
    int ax = 0;
    for (int d = 1; d < dim; ++d)
        if (mx[d] - mn[d] > mx[ax] - mn[ax]) ax = d;
    const int mid = lo + (hi - lo) / 2;
    std::nth_element(ids.begin() + lo, ids.begin() + mid, ids.begin() + hi, [&](int a, int b) {
        const double xa = xyz[size_t(a) * dim + ax], xb = xyz[size_t(b) * dim + ax];
        return xa < xb || (xa == xb && a < b);
    });
    rcb(ids, lo, mid, xyz, dim, maxsz, part, np);
    rcb(ids, mid, hi, xyz, dim, maxsz, part, np);
}

}  // namespace

void build_p1_patches(HostMesh &hm, int l, int target_blocks) {
    HostLevel &F = hm.levels[l];
    const HostLevel &C = hm.levels[l + 1];
    HostPatches &P = F.patch;
    P = HostPatches{};
    const int W = F.width, nf = F.nv, nc = C.nv;
    // about target_blocks patches, each of 16 to 128 coarse vertices (so that a
    // patch's rows fit one block of at most 1024 threads)
    const int maxsz = std::min(128, std::max(16, (nc + target_blocks - 1) / target_blocks));
    std::vector<int> ids(nc), part(nc, -1);
    for (int c = 0; c < nc; ++c) ids[c] = c;
    int nb = 0;
    rcb(ids, 0, nc, C.vxyz, C.vdim, maxsz, part, nb);
    P.nb = nb;
    std::vector<std::vector<int>> members(nb);
    for (int c = 0; c < nc; ++c) members[part[c]].push_back(c);            // ascending ids per patch
    std::vector<std::vector<int>> owned(nb);
    for (int v = 0; v < nf; ++v) owned[part[C.parent[2 * v]]].push_back(v);
    std::vector<int> slot(nf, -1);
    // rows first (ascending), then their neighbours not among them (ascending)
    auto ring = [&](const std::vector<int> &rows, std::vector<int> &out) {
        out = rows;
        for (size_t i = 0; i < rows.size(); ++i) slot[rows[i]] = int(i);
        std::vector<int> halo;
        for (int v : rows)
            for (int q = 0; q < W; ++q) {
                const int u = F.col[size_t(v) * W + q];
                if (slot[u] < 0) { slot[u] = -2; halo.push_back(u); }
            }
        std::sort(halo.begin(), halo.end());
        for (size_t i = 0; i < halo.size(); ++i) slot[halo[i]] = int(rows.size() + i);
        out.insert(out.end(), halo.begin(), halo.end());
    };
    P.f_ptr.push_back(0); P.c_ptr.push_back(0); P.cc_ptr.push_back(0); P.g_ptr.push_back(0);
    std::vector<int> set;
    for (int b = 0; b < nb; ++b) {
        // going down: children of the patch's coarse vertices, then their neighbours
        std::vector<int> f0;
        for (int c : members[b])
            for (int k = C.child_ptr[c]; k < C.child_ptr[c + 1]; ++k) f0.push_back(C.child_idx[k]);
        std::sort(f0.begin(), f0.end());
        f0.erase(std::unique(f0.begin(), f0.end()), f0.end());
        ring(f0, set);
        P.f0_base.push_back(int(P.lcol.size() / W));
        for (int v : f0)
            for (int q = 0; q < W; ++q) P.lcol.push_back(slot[F.col[size_t(v) * W + q]]);
        for (int c : members[b]) {
            P.c_ids.push_back(c);
            for (int k = C.child_ptr[c]; k < C.child_ptr[c + 1]; ++k) {
                P.cc_slot.push_back(slot[C.child_idx[k]]);
                P.cc_w.push_back(C.child_w[k]);
            }
            P.cc_ptr.push_back(int(P.cc_slot.size()));
        }
        P.c_ptr.push_back(int(P.c_ids.size()));
        P.f_n0.push_back(int(f0.size()));
        P.f_ids.insert(P.f_ids.end(), set.begin(), set.end());
        for (int v : set) P.fcol.insert(P.fcol.end(), F.col.begin() + size_t(v) * W, F.col.begin() + size_t(v + 1) * W);
        P.f_ptr.push_back(int(P.f_ids.size()));
        P.max_f0 = std::max(P.max_f0, int(f0.size()));
        P.max_f1 = std::max(P.max_f1, int(set.size()));
        for (int v : set) slot[v] = -1;
        // going up: owned fine vertices, then their neighbours
        ring(owned[b], set);
        P.g0_base.push_back(int(P.glcol.size() / W));
        for (int v : owned[b])
            for (int q = 0; q < W; ++q) P.glcol.push_back(slot[F.col[size_t(v) * W + q]]);
        P.g_nown.push_back(int(owned[b].size()));
        P.g_ids.insert(P.g_ids.end(), set.begin(), set.end());
        for (int v : set) {
            for (int q = 0; q < W; ++q) {
                const int j = F.col[size_t(v) * W + q];
                P.gcol.push_back(j);
                P.gpar.push_back(C.parent[2 * j]);
                P.gpar.push_back(C.parent[2 * j + 1]);
            }
            P.grow_par.push_back(C.parent[2 * v]);
            P.grow_par.push_back(C.parent[2 * v + 1]);
        }
        P.g_ptr.push_back(int(P.g_ids.size()));
        P.max_g1 = std::max(P.max_g1, int(set.size()));
        for (int v : set) slot[v] = -1;
    }
}

}  // namespace hdg
