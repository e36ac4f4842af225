// FP64 storage and arithmetic: the debug path. This translation unit is built
// with -fmad=false, so every multiply and add rounds separately, in the order
// written, as in the FP64 CPU oracle; division and square root are IEEE.
#include "lbm_launch.cuh"

namespace lbm {
const KernelTable kTableF64 = make_table<double>();
const KernelTable kTableF64Q7 = make_table7<double>();
} // namespace lbm
