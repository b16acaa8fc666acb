// Host-side layout of the single-CTA coarse cycle's shared memory (the tail
// image of k_p1.cu): a table of sizes and offsets per level, every level's
// staged arrays (ELL values, inverse diagonal, ELL columns and, below the
// first tail level, restriction weights, child pointers, child indices and
// parents), the coarsest level's FP64 inverse when it fits, then the scratch
// vectors.  The ELL values are staged slot-major (slot q of row i at
// q * nv + i) and the ELL columns as 16-bit indices, row-major, so that the
// kernel's shared-memory reads of a row are free of bank conflicts.  Kept apart from the CUDA code so that it can be checked on the CPU.
#include "common.h"

namespace hdg {

bool tail_layout(const std::vector<TailLevelSize> &lv, size_t tsz, size_t nc, TailLayout &out) {
    auto pad = [](size_t b) { return (b + 15) / 16 * 16; };
    const int n = int(lv.size());
    out = TailLayout{};
    out.hdr.assign(size_t(n), TailHdr{});
    size_t off = pad(sizeof(TailHdr) * size_t(n));
    auto put = [&](int32_t &o, int level, int kind, size_t bytes) {
        o = int32_t(off);
        if (bytes) out.pieces.push_back({off, pad(bytes), level, kind});
        off += pad(bytes);
    };
    for (int k = 0; k < n; ++k) {
        const TailLevelSize &L = lv[size_t(k)];
        const bool top = k == 0;
        TailHdr &H = out.hdr[size_t(k)];
        H.nv = L.nv;
        H.nnz = L.nnz;
        H.nci = top ? 0 : L.nci;
        H.W = L.W;
        put(H.oA, k, kTailA, tsz * size_t(L.nnz));
        put(H.oD, k, kTailD, tsz * size_t(L.nv));
        put(H.ocol, k, kTailCol, 2 * size_t(L.nnz));      // 16-bit columns
        if (!top) {
            put(H.ocw, k, kTailCw, tsz * size_t(L.nci));
            put(H.ocp, k, kTailCp, 4 * size_t(L.nv + 1));
            put(H.oci, k, kTailCi, 4 * size_t(L.nci));
            put(H.opar, k, kTailPar, 4 * size_t(2 * L.nfin));
        }
    }
    const size_t data_end = off;
    size_t scratch = 0;
    for (int k = 0; k < n; ++k) scratch += 4 * pad(tsz * size_t(lv[size_t(k)].nv));
    const size_t inv_bytes = pad(sizeof(double) * nc * nc);
    if (nc > 0 && inv_bytes <= kTailInvSmemMax && data_end + inv_bytes + scratch <= kTailSmemMax) {
        out.inv_off = int32_t(off);
        out.pieces.push_back({off, inv_bytes, n - 1, kTailInv});
        off += inv_bytes;
    }
    out.img_bytes = off;
    for (int k = 0; k < n; ++k) {
        const size_t v = pad(tsz * size_t(lv[size_t(k)].nv));
        TailHdr &H = out.hdr[size_t(k)];
        H.ox = int32_t(off); off += v;
        H.ox2 = int32_t(off); off += v;
        H.ob = int32_t(off); off += v;
        H.orr = int32_t(off); off += v;
    }
    out.smem_bytes = off;
    return off <= kTailSmemMax;
}

}  // namespace hdg
