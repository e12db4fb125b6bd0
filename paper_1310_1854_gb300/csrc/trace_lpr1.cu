// Instantiations of the traversal kernel for 1 lane(s) per ray.
#include "kernels.h"
#include "trace.cuh"

namespace vg {

void kernel_table_lpr1(KernelSet &k) {
    k.fn[0][MODE_TAU] = (const void *)trace_kernel<1, false, MODE_TAU, false>;
    k.fn[0][MODE_SEGS] = (const void *)trace_kernel<1, false, MODE_SEGS, false>;
    k.fn[0][MODE_GRAD] = (const void *)trace_kernel<1, false, MODE_GRAD, false>;
    k.fn[1][MODE_TAU] = (const void *)trace_kernel<1, true, MODE_TAU, false>;
    k.fn[1][MODE_SEGS] = (const void *)trace_kernel<1, true, MODE_SEGS, false>;
    k.fn[1][MODE_GRAD] = nullptr;
    k.fn[0][MODE_INTERACT] = (const void *)trace_kernel<1, false, MODE_INTERACT, false>;
    k.fn[1][MODE_INTERACT] = nullptr;
    k.fn[2][MODE_TAU] = (const void *)trace_kernel<1, false, MODE_TAU, false, true>;
    k.fn[2][MODE_SEGS] = (const void *)trace_kernel<1, false, MODE_SEGS, false, true>;
    k.batch = (const void *)trace_kernel<1, false, MODE_TAU, true>;
}

}  // namespace vg
