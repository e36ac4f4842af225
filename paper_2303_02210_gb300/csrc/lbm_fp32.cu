// FP32 storage and arithmetic: the fast path.
#include "lbm_launch.cuh"
#include "lbm_update7_tma.cuh"
#include "lbm_update_tma.cuh"

namespace lbm {
const KernelTable kTableF32 = make_table<float>(&prepare_update_tma<float>, &launch_update_tma<float>);
const KernelTable kTableF32Q7 = make_table7<float>(&prepare_update7_tma_any, &launch_update7_tma_any);

// the D2Q7 kernel's grid and tiles are sized by variant 0's figures
static_assert(TMA7_TY == tma_rows(0) && TMA7_CTAS == tma_ctas_per_sm(0), "D2Q7 TMA form = variant 0's tiles");

int launch_update_tma_ctas(int nsm, int variant) { return tma_ctas_per_sm(variant) * nsm; }

int launch_update_tma_rows(int variant) { return tma_rows(variant); }
} // namespace lbm
