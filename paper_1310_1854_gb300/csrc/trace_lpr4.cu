// Instantiations of the traversal kernel for 4 lane(s) per ray.
#include "kernels.h"
#include "trace.cuh"

namespace vg {

void kernel_table_lpr4(KernelSet &k) {
    k.fn[0][MODE_TAU] = (const void *)trace_kernel<4, false, MODE_TAU, false>;
    k.fn[0][MODE_SEGS] = (const void *)trace_kernel<4, false, MODE_SEGS, false>;
    k.fn[0][MODE_GRAD] = (const void *)trace_kernel<4, false, MODE_GRAD, false>;
    k.fn[1][MODE_TAU] = (const void *)trace_kernel<4, true, MODE_TAU, false>;
    k.fn[1][MODE_SEGS] = (const void *)trace_kernel<4, true, MODE_SEGS, false>;
    k.fn[1][MODE_GRAD] = nullptr;
    k.fn[0][MODE_INTERACT] = (const void *)trace_kernel<4, false, MODE_INTERACT, false>;
    k.fn[1][MODE_INTERACT] = nullptr;
    k.batch = (const void *)trace_kernel<4, false, MODE_TAU, true>;
}

}  // namespace vg
