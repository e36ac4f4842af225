// Launchers of one storage type, collected in the table the C ABI dispatches
// through.
#pragma once

#include "lbm_kernels.cuh"
#include "lbm_plan.cuh"

namespace lbm {

template <typename R>
struct Launch {
    static constexpr int UPD_TPB = 128;
    static constexpr int UPD_NR = sizeof(R) == 4 ? 2 : 1;

    static cudaError_t fill(const SimDev &d, cudaStream_t s)
    {
        k_fill<R><<<4 * 152, 256, 0, s>>>(d);
        return cudaGetLastError();
    }
    static cudaError_t ghosts(const SimDev &d, cudaStream_t s)
    {
        k_ghosts<R><<<152, 256, 0, s>>>(d);
        return cudaGetLastError();
    }
    static cudaError_t scan(const SimDev &d, int cur, cudaStream_t s)
    {
        k_scan<R><<<4 * 152, 256, 0, s>>>(d, cur);
        return cudaGetLastError();
    }
    static cudaError_t plan(const SimDev &d, int init, cudaStream_t s)
    {
        return launch_plan<R>(d, init, s);
    }
    static cudaError_t inject(const SimDev &d, cudaStream_t s)
    {
        k_inject<R><<<152, 128, 0, s>>>(d);
        return cudaGetLastError();
    }
    static cudaError_t update(const SimDev &d, cudaStream_t s)
    {
        k_update<R, UPD_TPB, UPD_NR><<<d.update_grid, UPD_TPB, 0, s>>>(d);
        return cudaGetLastError();
    }
    static cudaError_t fields(const SimDev &d, int cur, double *rho, double *ux, double *uy, cudaStream_t s)
    {
        k_fields<R><<<4 * 152, 256, 0, s>>>(d, cur, rho, ux, uy);
        return cudaGetLastError();
    }
    static int update_blocks_per_sm()
    {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_update<R, UPD_TPB, UPD_NR>, UPD_TPB, 0) != cudaSuccess)
            return 0;
        return n;
    }
};

template <typename R>
constexpr KernelTable make_table()
{
    return KernelTable{(int)sizeof(R),       &Launch<R>::fill,          &Launch<R>::ghosts,
                       &Launch<R>::scan,     &Launch<R>::plan,          &Launch<R>::inject,
                       &Launch<R>::update,
                       &Launch<R>::fields,   &plan_blocks_per_sm<R>,    &Launch<R>::update_blocks_per_sm,
                       Launch<R>::UPD_TPB};
}

} // namespace lbm
