// FP32 storage and arithmetic: the fast path.
#include "lbm_launch.cuh"
#include "lbm_update_tma.cuh"

namespace lbm {
const KernelTable kTableF32 = make_table<float>(&prepare_update_tma<float>, &launch_update_tma<float>);
const KernelTable kTableF32Q7 = make_table7<float>();

int launch_update_tma_ctas(int nsm, int variant) { return tma_ctas_per_sm(variant) * nsm; }

int launch_update_tma_rows(int variant) { return tma_rows(variant); }
} // namespace lbm
