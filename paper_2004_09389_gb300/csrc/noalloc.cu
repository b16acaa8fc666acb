// Step 1 (condensed right-hand side) without any device allocation.
//
// hdg_condensed_rhs_dev keeps its per-cell partial results in the handle's
// solver workspace.  hdg_condensed_rhs_noalloc_dev computes exactly the same
// thing with that scratch in a fixed array that lives in this library's
// device image instead, so the call itself never allocates.
#include "common.h"

#include <mutex>

namespace {

// Scratch: the per-cell products W_K r_K (n_cells * 3(p+1) doubles) followed by
// the right-hand side in the internal node-major layout (n_facets * (p+1)).
constexpr size_t kScratchDoubles = size_t(1) << 22;      // 32 MiB
static __device__ __align__(256) double g_rhs_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double *g_scratch_addr[kMaxDevices] = {};

// Device address of g_rhs_scratch on the current device (looked up once per device).
cudaError_t scratch_address(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_rhs_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

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
    double *scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) {
        h->err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return HDG_ECUDA;
    }
    // every scratch entry read by the gather is written first by the cell kernel:
    // nothing has to start at zero
    double *ycell = scratch, *g_int = scratch + cell_part;
    e = hdg::launch_rhs(h, r_u, r_h, g_int, ycell);
    if (e == cudaSuccess) e = hdg::launch_to_external(h, g_int, g);
    if (e != cudaSuccess) {
        h->err = std::string("hdg_condensed_rhs_noalloc_dev: ") + cudaGetErrorString(e);
        return HDG_ECUDA;
    }
    return HDG_OK;
}
