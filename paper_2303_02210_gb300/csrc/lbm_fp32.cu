// FP32 storage and arithmetic: the fast path.
#include "lbm_kernels.cuh"

namespace lbm {
const KernelTable kTableF32 = make_table<float>();
} // namespace lbm
