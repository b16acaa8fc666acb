// Host-side check of the P1 patches that the fused smoothing kernels use
// (built by build_host_mesh, csrc/mesh.cpp): every index the kernels follow
// is recomputed here from the level operators and transfers and compared.
// Compiled with the library's mesh sources by tests/test_p1_patches.py.
#include "common.h"

#include <cstdio>
#include <string>

using namespace hdg;

extern "C" int check_patches(const hdg_mesh_desc *d, char *out, int len) {
    HostMesh hm;
    const std::string e = build_host_mesh(d, hm);
    if (!e.empty()) {
        snprintf(out, len, "mesh: %s", e.c_str());
        return 1;
    }
    std::string rep;
    int bad = 0;
    auto fail = [&](const std::string &m) { ++bad; rep += "BAD " + m + "\n"; };
    for (size_t l = 0; l + 1 < hm.levels.size(); ++l) {
        const HostLevel &F = hm.levels[l], &C = hm.levels[l + 1];
        const HostPatches &P = F.patch;
        const int W = F.width, nb = P.nb;
        if (F.nv > kPatchMaxVertices) {
            if (nb != 0) fail("patches on a level above the size limit");
            continue;
        }
        if (nb <= 0) { fail("no patches"); continue; }
        const std::string lv = "level " + std::to_string(l) + ": ";
        std::vector<int> cseen(C.nv, 0), fcov(F.nv, 0), own(F.nv, 0);
        int m1 = 0, m0 = 0, mg = 0;
        for (int b = 0; b < nb; ++b) {
            const int s0 = P.f_ptr[b], n1 = P.f_ptr[b + 1] - s0, n0 = P.f_n0[b], r0 = P.f0_base[b];
            if (n0 <= 0 || n0 > n1) fail(lv + "F0 size");
            m1 = std::max(m1, n1);
            m0 = std::max(m0, n0);
            for (int s = 0; s < n0; ++s) {
                const int v = P.f_ids[s0 + s];
                fcov[v]++;
                for (int q = 0; q < W; ++q) {
                    const int ls = P.lcol[size_t(r0 + s) * W + q];
                    if (ls < 0 || ls >= n1 || P.f_ids[s0 + ls] != F.col[size_t(v) * W + q]) { fail(lv + "lcol"); break; }
                }
            }
            if (P.c_ptr[b + 1] - P.c_ptr[b] > n0) fail(lv + "more coarse vertices than F0 rows");
            for (int c = P.c_ptr[b]; c < P.c_ptr[b + 1]; ++c) {
                const int cid = P.c_ids[c];
                cseen[cid]++;
                if (P.cc_ptr[c + 1] - P.cc_ptr[c] != C.child_ptr[cid + 1] - C.child_ptr[cid]) fail(lv + "child count");
                for (int k = P.cc_ptr[c], kk = C.child_ptr[cid]; k < P.cc_ptr[c + 1]; ++k, ++kk) {
                    const int sl = P.cc_slot[k];
                    if (sl < 0 || sl >= n0 || P.f_ids[s0 + sl] != C.child_idx[kk] || P.cc_w[k] != C.child_w[kk]) {
                        fail(lv + "child slot or weight");
                        break;
                    }
                }
            }
            const int g0 = P.g_ptr[b], ng = P.g_ptr[b + 1] - g0, no = P.g_nown[b], q0 = P.g0_base[b];
            mg = std::max(mg, ng);
            if (no > ng) fail(lv + "owned rows");
            for (int s = 0; s < no; ++s) {
                const int v = P.g_ids[g0 + s];
                own[v]++;
                for (int q = 0; q < W; ++q) {
                    const int ls = P.glcol[size_t(q0 + s) * W + q];
                    if (ls < 0 || ls >= ng || P.g_ids[g0 + ls] != F.col[size_t(v) * W + q]) { fail(lv + "glcol"); break; }
                }
            }
        }
        if (P.fcol.size() != P.f_ids.size() * W || P.gcol.size() != P.g_ids.size() * W ||
            P.gpar.size() != 2 * P.g_ids.size() * W || P.grow_par.size() != 2 * P.g_ids.size())
            fail(lv + "copy sizes");
        for (size_t r = 0; r < P.f_ids.size(); ++r)
            for (int q = 0; q < W; ++q)
                if (P.fcol[r * W + q] != F.col[size_t(P.f_ids[r]) * W + q]) { fail(lv + "fcol"); r = P.f_ids.size(); break; }
        for (size_t r = 0; r < P.g_ids.size(); ++r) {
            const int v = P.g_ids[r];
            if (P.grow_par[2 * r] != C.parent[2 * v] || P.grow_par[2 * r + 1] != C.parent[2 * v + 1]) { fail(lv + "grow_par"); break; }
            bool ok = true;
            for (int q = 0; q < W && ok; ++q) {
                const int j = F.col[size_t(v) * W + q];
                ok = P.gcol[r * W + q] == j && P.gpar[(r * W + q) * 2] == C.parent[2 * j] &&
                     P.gpar[(r * W + q) * 2 + 1] == C.parent[2 * j + 1];
            }
            if (!ok) { fail(lv + "gcol / gpar"); break; }
        }
        for (int c = 0; c < C.nv; ++c)
            if (cseen[c] != 1) { fail(lv + "coarse vertex not in exactly one patch"); break; }
        for (int v = 0; v < F.nv; ++v)
            if (fcov[v] < 1) { fail(lv + "fine vertex in no F0"); break; }
        for (int v = 0; v < F.nv; ++v)
            if (own[v] != 1) { fail(lv + "fine vertex not owned exactly once"); break; }
        if (m1 != P.max_f1 || m0 != P.max_f0 || mg != P.max_g1) fail(lv + "maximum sizes");
        char buf[160];
        snprintf(buf, sizeof buf, "level %zu: %d -> %d vertices, %d patches, max F1 %d, max up rows %d\n", l, F.nv,
                 C.nv, nb, P.max_f1, P.max_g1);
        rep += buf;
    }
    snprintf(out, len, "%s", rep.c_str());
    return bad ? 2 : 0;
}
