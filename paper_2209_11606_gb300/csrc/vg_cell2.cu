// 2D cell kernel (polygon cells); see vg_cell3.cu for the 3D method.
#include "vg_internal.cuh"

namespace vg {

cudaError_t launch_cells2(const Grid &, const Store &, const Out &, const Params &, const Offsets &, int,
                          unsigned *, int, int, const int *, int, int, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace vg
