// FP32 storage and arithmetic: the fast path.
#include "lbm_launch.cuh"
#include "lbm_update_tma.cuh"

namespace lbm {
const KernelTable kTableF32 = make_table<float>();


cudaError_t launch_update_tma_f32(const SimDev &d, int cur, uint32_t t, const CUtensorMap *maps, int nsm,
                                  int variant, cudaStream_t s)
{
    return launch_update_tma(d, cur, t, maps, nsm, variant, s);
}

int launch_update_tma_ctas(int nsm, int variant) { return tma_ctas_per_sm(variant) * nsm; }

int launch_update_tma_rows(int variant) { return tma_rows(variant); }
} // namespace lbm
