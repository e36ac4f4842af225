// 16-bit population storage (FP16 and BF16, the deviation from the rest state
// of density rho_init) with FP32 arithmetic: half the bytes per node update
// of the FP32 path, on the same update kernels.
#include "lbm_launch.cuh"
#include "lbm_update_tma.cuh"
#include "lbm_update_tma_batch.cuh"

namespace lbm {
const KernelTable kTableF16 =
    make_table<__half>(&prepare_update_tma<__half>, &launch_update_tma<__half>, &tile_variant_info<__half>,
                       &launch_update_tma_batch<__half>);
const KernelTable kTableBF16 = make_table<__nv_bfloat16>(&prepare_update_tma<__nv_bfloat16>,
                                                         &launch_update_tma<__nv_bfloat16>,
                                                         &tile_variant_info<__nv_bfloat16>,
                                                         &launch_update_tma_batch<__nv_bfloat16>);
} // namespace lbm
