// Launchers of one population storage type (float, double, __half or
// __nv_bfloat16), collected in the table the C ABI dispatches
// through.
#pragma once

#include "lbm_d2q7.cuh"
#include "lbm_kernels.cuh"
#include "lbm_plan.cuh"

namespace lbm {

template <typename S>
struct Launch {
    static constexpr int UPD_TPB = 128;
    static constexpr int UPD_NR = sizeof(S) == 8 ? 1 : 2;

    static cudaError_t fill(const SimDev &d, cudaStream_t s)
    {
        k_fill<S><<<4 * 152, 256, 0, s>>>(d);
        return cudaGetLastError();
    }
    static cudaError_t ghosts(const SimDev &d, cudaStream_t s)
    {
        k_ghosts<S><<<152, 256, 0, s>>>(d);
        return cudaGetLastError();
    }
    static cudaError_t scan(const SimDev &d, int cur, cudaStream_t s)
    {
        k_scan<S><<<4 * 152, 256, 0, s>>>(d, cur);
        return cudaGetLastError();
    }
    static cudaError_t plan(const SimDev &d, int init, cudaStream_t s)
    {
        return launch_plan<S>(d, init, s);
    }
    static cudaError_t inject(const SimDev &d, cudaStream_t s)
    {
        k_inject<S><<<152, 128, 0, s>>>(d);
        return cudaGetLastError();
    }
    static cudaError_t update(const SimDev &d, cudaStream_t s)
    {
        k_update<S, UPD_TPB, UPD_NR><<<d.update_grid, UPD_TPB, 0, s>>>(d);
        return cudaGetLastError();
    }
    static cudaError_t fields(const SimDev &d, int cur, double *rho, double *ux, double *uy, cudaStream_t s)
    {
        k_fields<S><<<4 * 152, 256, 0, s>>>(d, cur, rho, ux, uy);
        return cudaGetLastError();
    }
    static cudaError_t batch_inject(const SimDev *ds, int nslots, int grid, cudaStream_t s)
    {
        k_inject_batch<S><<<grid, INJ_NT, 0, s>>>(ds, nslots);
        return cudaGetLastError();
    }
    static cudaError_t batch_update(const SimDev *ds, const int4 *bm, int nb, cudaStream_t s)
    {
        k_update_batch<S, UPD_TPB, UPD_NR><<<nb, UPD_TPB, 0, s>>>(ds, bm);
        return cudaGetLastError();
    }
    static cudaError_t batch_plan(const SimDev *ds, int nslots, int cap, cudaStream_t s)
    {
        return launch_plan_batch<S>(ds, nslots, cap, s);
    }
    static int update_blocks_per_sm()
    {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_update<S, UPD_TPB, UPD_NR>, UPD_TPB, 0) != cudaSuccess)
            return 0;
        return n;
    }
};

template <typename S>
constexpr KernelTable make_table(cudaError_t (*tma_prepare)(const SimDev &, int) = nullptr,
                                 cudaError_t (*tma_update)(const SimDev &, const CUtensorMap *, int, bool,
                                                           cudaStream_t) = nullptr,
                                 int (*tma_info)(int, int *, int *, int *) = nullptr,
                                 cudaError_t (*batch_update_tma)(const SimDev *, const MemberConst *,
                                                                 const CUtensorMap *, int, int, int, int,
                                                                 cudaStream_t) = nullptr)
{
    return KernelTable{(int)sizeof(S),       &Launch<S>::fill,          &Launch<S>::ghosts,
                       &Launch<S>::scan,     &Launch<S>::plan,          &Launch<S>::inject,
                       &Launch<S>::update,
                       &Launch<S>::fields,   &plan_blocks_per_sm<S>,    &Launch<S>::update_blocks_per_sm,
                       Launch<S>::UPD_TPB,   tma_prepare,               tma_update,        tma_info,
                       &Launch<S>::batch_inject, &Launch<S>::batch_update, &Launch<S>::batch_plan,
                       batch_update_tma};
}

// The triangular D2Q7 lattice (FP32 or FP64 storage; the TMA-staged update
// for FP32 comes with the table).
template <typename S>
struct Launch7 {
    static constexpr int UPD_TPB = 128;
    static constexpr int UPD_NR = sizeof(S) == 8 ? 1 : 2;

    static cudaError_t fill(const SimDev &d, cudaStream_t s)
    {
        k_fill7<S><<<4 * 152, 256, 0, s>>>(d);
        return cudaGetLastError();
    }
    static cudaError_t ghosts(const SimDev &d, cudaStream_t s)
    {
        k_ghosts7<S><<<152, 256, 0, s>>>(d);
        return cudaGetLastError();
    }
    static cudaError_t scan(const SimDev &d, int cur, cudaStream_t s)
    {
        k_scan7<S><<<4 * 152, 256, 0, s>>>(d, cur);
        return cudaGetLastError();
    }
    static cudaError_t plan(const SimDev &d, int init, cudaStream_t s)
    {
        return launch_plan<S, Lat7>(d, init, s);
    }
    static cudaError_t inject(const SimDev &d, cudaStream_t s)
    {
        k_inject<S, Lat7><<<152, 128, 0, s>>>(d);
        return cudaGetLastError();
    }
    static cudaError_t update(const SimDev &d, cudaStream_t s)
    {
        k_update7<S, UPD_TPB, UPD_NR><<<d.update_grid, UPD_TPB, 0, s>>>(d);
        return cudaGetLastError();
    }
    static cudaError_t fields(const SimDev &d, int cur, double *rho, double *ux, double *uy, cudaStream_t s)
    {
        k_fields7<S><<<4 * 152, 256, 0, s>>>(d, cur, rho, ux, uy);
        return cudaGetLastError();
    }
    static cudaError_t batch_inject(const SimDev *ds, int nslots, int grid, cudaStream_t s)
    {
        k_inject_batch<S, Lat7><<<grid, INJ_NT, 0, s>>>(ds, nslots);
        return cudaGetLastError();
    }
    static cudaError_t batch_update(const SimDev *ds, const int4 *bm, int nb, cudaStream_t s)
    {
        k_update7_batch<S, UPD_TPB, UPD_NR><<<nb, UPD_TPB, 0, s>>>(ds, bm);
        return cudaGetLastError();
    }
    static cudaError_t batch_plan(const SimDev *ds, int nslots, int cap, cudaStream_t s)
    {
        return launch_plan_batch<S, Lat7>(ds, nslots, cap, s);
    }
    static int update_blocks_per_sm()
    {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_update7<S, UPD_TPB, UPD_NR>, UPD_TPB, 0) !=
            cudaSuccess)
            return 0;
        return n;
    }
};

// (tma_prepare, tma_update: the TMA-staged update of lbm_update7_tma.cuh for
// FP32 storage, null otherwise)
template <typename S>
constexpr KernelTable make_table7(cudaError_t (*tma_prepare)(const SimDev &, int) = nullptr,
                                  cudaError_t (*tma_update)(const SimDev &, const CUtensorMap *, int, bool,
                                                            cudaStream_t) = nullptr,
                                  int (*tma_info)(int, int *, int *, int *) = nullptr)
{
    return KernelTable{(int)sizeof(S),         &Launch7<S>::fill,          &Launch7<S>::ghosts,
                       &Launch7<S>::scan,      &Launch7<S>::plan,          &Launch7<S>::inject,
                       &Launch7<S>::update,    &Launch7<S>::fields,        &plan_blocks_per_sm<S, Lat7>,
                       &Launch7<S>::update_blocks_per_sm,
                       Launch7<S>::UPD_TPB,    tma_prepare,                tma_update,        tma_info,
                       &Launch7<S>::batch_inject, &Launch7<S>::batch_update, &Launch7<S>::batch_plan,
                       nullptr};
}

} // namespace lbm
