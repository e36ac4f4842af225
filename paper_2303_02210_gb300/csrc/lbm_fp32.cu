// FP32 storage and arithmetic: the fast path.
#include "lbm_launch.cuh"
#include "lbm_update_tma.cuh"

namespace lbm {
const KernelTable kTableF32 = make_table<float>();


cudaError_t prepare_update_tma_f32(const SimDev &d, int variant) { return prepare_update_tma(d, variant); }

cudaError_t launch_update_tma_f32(const SimDev &d, const CUtensorMap *maps, int variant, bool pdl, cudaStream_t s)
{
    return launch_update_tma(d, maps, variant, pdl, s);
}

int launch_update_tma_ctas(int nsm, int variant) { return tma_ctas_per_sm(variant) * nsm; }

int launch_update_tma_rows(int variant) { return tma_rows(variant); }
} // namespace lbm
