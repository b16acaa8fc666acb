// Step 1 (condensed right-hand side) without any device allocation.
//
// hdg_condensed_rhs_dev keeps its per-cell partial results in the handle's
// solver workspace.  hdg_condensed_rhs_noalloc_dev computes exactly the same
// thing with that scratch in a fixed array that lives in this library's
// device image instead, so the call itself never allocates.
//
// The library is linked from separate objects, so this file is a module of
// its own; under lazy module loading the array is only placed on a device
// when something first touches the module.  hdg_setup does that
// (noalloc_prepare), so that the entry point never triggers the load.
#include "common.h"

namespace {

// Scratch: the per-cell products W_K r_K (n_cells * 3(p+1) doubles, rounded
// up to 32) followed by the right-hand side in the internal node-major layout
// (n_facets * (p+1)).
constexpr size_t kScratchDoubles = size_t(1) << 22;      // 32 MiB
static __device__ __align__(256) double g_rhs_scratch[kScratchDoubles];

}  // namespace

// Called by hdg_setup with the handle's device current: loads this module on
// that device (if it is not loaded yet) and keeps the array's device address
// in the handle.  In host code g_rhs_scratch is only a host-side stand-in, so
// the address must come from cudaGetSymbolAddress.
cudaError_t hdg::noalloc_prepare(hdg_handle *h) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_rhs_scratch);
    if (e != cudaSuccess) return e;
    h->noalloc_scratch = static_cast<double *>(p);
    return cudaSuccess;
}

extern "C" int hdg_condensed_rhs_noalloc_dev(hdg_handle *h, const double *r_u, const double *r_h, double *g) {
    if (!h) return HDG_EINVAL;
    if (!r_u || !r_h || !g) {
        h->err = "NULL pointer argument";
        return HDG_EINVAL;
    }
    const size_t cell_part = (size_t(h->N) * size_t(h->m) + 31) / 32 * 32;   // keep the second part 256-B aligned
    const size_t need = cell_part + size_t(h->NT);
    if (need > kScratchDoubles) {
        h->err = "hdg_condensed_rhs_noalloc_dev: needs " + std::to_string(need) +
                 " doubles of scratch (n_cells * 3(p+1) + n_facets * (p+1)), more than the fixed " +
                 std::to_string(kScratchDoubles);
        return HDG_EINVAL;
    }
    if (!h->condensed) {
        h->err = "hdg_condense has not run on this handle";
        return HDG_ESTATE;
    }
    if (!h->noalloc_scratch) {
        h->err = "hdg_condensed_rhs_noalloc_dev: the scratch address was not resolved at set-up";
        return HDG_ESTATE;
    }
    // every scratch entry read by the gather is written first by the cell kernel
    // of the same call: nothing has to start at zero
    double *ycell = h->noalloc_scratch, *g_int = h->noalloc_scratch + cell_part;
    cudaError_t e = hdg::account_launch(h, HDG_PROF_RHS, 2, [&]() { return hdg::launch_rhs(h, r_u, r_h, g_int, ycell); });
    if (e == cudaSuccess)
        e = hdg::account_launch(h, HDG_PROF_LAYOUT, 1, [&]() { return hdg::launch_to_external(h, g_int, g); });
    if (e != cudaSuccess) {
        h->err = std::string("hdg_condensed_rhs_noalloc_dev: ") + cudaGetErrorString(e);
        return HDG_ECUDA;
    }
    return HDG_OK;
}
