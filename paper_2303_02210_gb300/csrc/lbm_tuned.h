// Generated by paper_2303_02210_gb300/autotune.py; do not edit by hand.
// The update form (KernelTable::tma_info variant: 0 two-row tiles, 1
// four-row tiles, 2 two-row tiles with bulk tensor stores) and the planner's
// cooperative grid (0: the width/capacity rule) with the shortest step, per
// storage type (LBM_FP32 0, LBM_FP16 2, LBM_BF16 3) and lattice width.
// Measured on NVIDIA GB300, 2026-12-04: whole steps of the
// benchmark's lattice shape at each width, timed by CUDA events.
#pragma once

namespace lbm {
struct TunedShape {
    int precision, width, variant, plan_blocks;
};
constexpr TunedShape kTunedShapes[] = {
    {0, 256, 0, 48}, // tma, 24.0 us per step
    {0, 512, 0, 48}, // tma, 24.6 us per step
    {0, 1024, 0, 4}, // tma, 24.6 us per step
    {0, 2048, 0, 38}, // tma, 32.5 us per step
    {0, 4096, 2, 64}, // tma_st, 72.2 us per step
    {0, 8192, 2, 64}, // tma_st, 217.4 us per step
    {2, 256, 0, 64}, // tma, 24.4 us per step
    {2, 512, 0, 4}, // tma, 24.6 us per step
    {2, 1024, 0, 24}, // tma, 26.8 us per step
    {2, 2048, 1, 16}, // tma1, 32.8 us per step
    {2, 4096, 1, 64}, // tma1, 70.2 us per step
    {2, 8192, 0, 64}, // tma, 206.8 us per step
    {3, 256, 0, 64}, // tma, 24.5 us per step
    {3, 512, 0, 4}, // tma, 24.6 us per step
    {3, 1024, 0, 24}, // tma, 26.8 us per step
    {3, 2048, 0, 16}, // tma, 32.9 us per step
    {3, 4096, 1, 64}, // tma1, 71.9 us per step
    {3, 8192, 0, 64}, // tma, 212.4 us per step
};
constexpr int kTunedShapeCount = (int)(sizeof(kTunedShapes) / sizeof(kTunedShapes[0]));
// batched form: FP32 members at least this wide (all of them) store in bulk
constexpr int kTunedBatchBulkMinWidth = 4096;
} // namespace lbm
