// Host-side check of the single-CTA coarse cycle's shared-memory layout
// (tail_layout, csrc/layout.cpp) on the levels of a real hierarchy: every
// admissible first tail level, FP64 and FP32 values.  Compiled with the
// library's host sources by tests/test_tail_layout.py.
#include "common.h"

#include <cstdio>
#include <string>

using namespace hdg;

extern "C" int check_tail_layouts(const hdg_mesh_desc *d, char *out, int len) {
    HostMesh hm;
    const std::string e = build_host_mesh(d, hm);
    if (!e.empty()) {
        snprintf(out, len, "mesh: %s", e.c_str());
        return 1;
    }
    auto pad = [](size_t b) { return (b + 15) / 16 * 16; };
    std::string rep;
    int bad = 0, checked = 0;
    auto fail = [&](const std::string &m) { ++bad; rep += "BAD " + m + "\n"; };
    const int nlev = int(hm.levels.size());
    const size_t nc = size_t(hm.levels.back().nv);
    for (int first = nlev - 1; first >= 0; --first) {
        if (hm.levels[first].nv > 4096 || nlev - first > kTailMaxLevels) break;
        std::vector<TailLevelSize> lv;
        for (int l = first; l < nlev; ++l) {
            const HostLevel &L = hm.levels[l];
            const bool top = l == first;
            lv.push_back({L.nv, int(L.col.size()), L.width, top ? 0 : int(L.child_idx.size()),
                          top ? 0 : hm.levels[l - 1].nv});
        }
        for (size_t tsz : {size_t(8), size_t(4)}) {
            ++checked;
            TailLayout lay;
            const bool ok = tail_layout(lv, tsz, nc, lay);
            const std::string tag = "first level " + std::to_string(first) + " tsz " + std::to_string(tsz) + ": ";
            if (ok != (lay.smem_bytes <= kTailSmemMax)) fail(tag + "return value");
            const size_t n = lv.size(), table = pad(sizeof(TailHdr) * n);
            if (lay.hdr.size() != n) fail(tag + "table size");
            if (lay.img_bytes % 16 || lay.smem_bytes % 16) fail(tag + "totals not 16-byte multiples");
            size_t at = table;
            for (const TailPiece &q : lay.pieces) {
                if (q.off % 16 || q.bytes % 16 || q.bytes == 0) fail(tag + "piece alignment");
                if (q.off < at) fail(tag + "pieces overlap or precede the table");
                at = q.off + q.bytes;
            }
            if (at != lay.img_bytes) fail(tag + "image end");
            auto find = [&](int level, int kind) -> const TailPiece * {
                for (const TailPiece &q : lay.pieces)
                    if (q.level == level && q.kind == kind) return &q;
                return nullptr;
            };
            for (size_t k = 0; k < n; ++k) {
                const TailHdr &H = lay.hdr[k];
                const TailLevelSize &L = lv[k];
                const int lvl = int(k);
                if (H.nv != L.nv || H.nnz != L.nnz || H.W != L.W || H.nci != (k ? L.nci : 0)) fail(tag + "table sizes");
                struct Want { int kind; int32_t off; size_t bytes; };
                std::vector<Want> want = {{kTailA, H.oA, tsz * L.nnz}, {kTailD, H.oD, tsz * L.nv},
                                          {kTailCol, H.ocol, 2 * size_t(L.nnz)}};
                if (k) {
                    want.push_back({kTailCw, H.ocw, tsz * L.nci});
                    want.push_back({kTailCp, H.ocp, 4 * size_t(L.nv + 1)});
                    want.push_back({kTailCi, H.oci, 4 * size_t(L.nci)});
                    want.push_back({kTailPar, H.opar, 4 * size_t(2 * L.nfin)});
                }
                for (const Want &w : want) {
                    const TailPiece *q = find(lvl, w.kind);
                    if (!q || size_t(w.off) != q->off || q->bytes != pad(w.bytes)) fail(tag + "table offset or piece size");
                }
                const size_t v = pad(tsz * size_t(L.nv));
                for (int32_t o : {H.ox, H.ox2, H.ob, H.orr})
                    if (size_t(o) < lay.img_bytes || size_t(o) + v > lay.smem_bytes || o % 16) fail(tag + "scratch vector");
                if (H.ox2 != H.ox + int32_t(v) || H.ob != H.ox2 + int32_t(v) || H.orr != H.ob + int32_t(v))
                    fail(tag + "scratch vectors overlap");
            }
            const size_t inv = pad(8 * nc * nc);
            const TailPiece *qi = find(int(n) - 1, kTailInv);
            size_t scratch = 0;
            for (const TailLevelSize &L : lv) scratch += 4 * pad(tsz * size_t(L.nv));
            const size_t data_end = lay.img_bytes - (qi ? qi->bytes : 0);
            const bool fits = inv <= kTailInvSmemMax && data_end + inv + scratch <= kTailSmemMax;
            if (bool(qi) != fits || (qi && (qi->bytes != inv || int32_t(qi->off) != lay.inv_off)) ||
                (!qi && lay.inv_off != -1))
                fail(tag + "inverse staging");
            char buf[200];
            snprintf(buf, sizeof buf, "first tail level %d (%d vertices), %zu-byte values: image %zu B, shared %zu B, inverse %s%s\n",
                     first, hm.levels[first].nv, tsz, lay.img_bytes, lay.smem_bytes, qi ? "staged" : "global",
                     ok ? "" : " (over the limit)");
            rep += buf;
        }
    }
    if (!checked) fail("no admissible tail start");
    snprintf(out, len, "%s", rep.c_str());
    return bad ? 2 : 0;
}
