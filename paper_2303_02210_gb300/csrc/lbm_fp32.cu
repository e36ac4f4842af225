// FP32 storage and arithmetic: the fast path.
#include "lbm_launch.cuh"
#include "lbm_update7_tma.cuh"
#include "lbm_update_tma.cuh"
#include "lbm_update_tma_batch.cuh"

namespace lbm {

// the D2Q7 lattice has one staged form: two-row tiles
static int update7_staged_info(int variant, int *box_rows, int *iter_rows, int *ctas_per_sm)
{
    if (variant != 0) return -1;
    *box_rows = TMA7_TY + 2;
    *iter_rows = TMA7_TY;
    *ctas_per_sm = TMA7_CTAS;
    return 0;
}

const KernelTable kTableF32 =
    make_table<float>(&prepare_update_tma<float>, &launch_update_tma<float>, &tile_variant_info<float>,
                      &launch_update_tma_batch<float>);
const KernelTable kTableF32Q7 =
    make_table7<float>(&prepare_update7_tma_any, &launch_update7_tma_any, &update7_staged_info);

} // namespace lbm
