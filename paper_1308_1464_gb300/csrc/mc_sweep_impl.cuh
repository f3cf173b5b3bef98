// mc_sweep_impl.cuh -- launch code of the fused step for one Riemann solver;
// included once per solver translation unit.
#pragma once

#include "mc_internal.h"
#include "mc_sweep.cuh"

namespace mc {

template <class RP>
cudaError_t sweep_launch_t(const SweepLaunch& L)
{
    using T = typename RP::real;
    SweepArgs<RP> a;
    a.rp.setup(L.prob.param, L.prob.efix);
    a.qa = static_cast<T*>(L.qa);
    a.qb = static_cast<T*>(L.qb);
    a.cur = L.cur_dev;
    a.dt_dev = L.dt_dev;
    a.dt = L.dt;
    a.dx = L.prob.dx;
    a.dy = L.prob.dy;
    a.mx = L.prob.mx;
    a.my = L.prob.my;
    a.ld_x = L.lay.ld_x;
    a.ld_field = L.lay.ld_field;
    a.x_offset = L.lay.x_offset;
    a.limiter = L.prob.limiter;
    a.order = L.prob.order;
    a.transverse = L.prob.transverse;
    a.tile_rows = L.tile_rows;
    a.ntasks = ntasks_for(L.prob, L.tile_rows, &a.nbands);
    a.smax_bits = L.smax_bits;
    a.status = L.status;

    constexpr int smem = sweep_smem_bytes(sizeof(T), RP::NEQ);
    int blocks = (a.ntasks + SWEEP_WARPS - 1) / SWEEP_WARPS;
    if (L.max_blocks > 0 && blocks > L.max_blocks) blocks = L.max_blocks;
    ctu_sweep_kernel<RP><<<blocks, SWEEP_WARPS * 32, smem, L.stream>>>(L.map_a, L.map_b, a);
    return cudaGetLastError();
}

// Raises the kernel's dynamic shared-memory limit; called once per context
// (outside any stream capture) before the first launch.
template <class RP>
cudaError_t sweep_prepare_t()
{
    using T = typename RP::real;
    constexpr int smem = sweep_smem_bytes(sizeof(T), RP::NEQ);
    return cudaFuncSetAttribute(ctu_sweep_kernel<RP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem);
}

template <class RP>
cudaError_t maxspeed_launch_t(const mc_problem& p, const mc_layout& lay, const void* q,
                              unsigned long long* out, cudaStream_t s)
{
    using T = typename RP::real;
    RP rp;
    rp.setup(p.param, p.efix);
    long long n = (long long)p.mx * p.my;
    int blocks = int((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    max_cell_speed_kernel<RP><<<blocks, 256, 0, s>>>(rp, static_cast<const T*>(q), p.mx, p.my,
                                                      lay.ld_x, lay.ld_field, lay.x_offset, p.dx,
                                                      p.dy, out);
    return cudaGetLastError();
}

}  // namespace mc

#define MC_DEFINE_SOLVER_LAUNCHERS(NAME, RPT)                                                  \
    namespace mc {                                                                             \
    cudaError_t sweep_launch_##NAME(const SweepLaunch& L)                                      \
    {                                                                                          \
        return L.prob.dtype == MC_F64 ? sweep_launch_t<RPT<double>>(L)                         \
                                      : sweep_launch_t<RPT<float>>(L);                         \
    }                                                                                          \
    cudaError_t sweep_prepare_##NAME(int dtype)                                                \
    {                                                                                          \
        return dtype == MC_F64 ? sweep_prepare_t<RPT<double>>() : sweep_prepare_t<RPT<float>>(); \
    }                                                                                          \
    cudaError_t maxspeed_launch_##NAME(const mc_problem& p, const mc_layout& lay,              \
                                       const void* q, unsigned long long* out, cudaStream_t s) \
    {                                                                                          \
        return p.dtype == MC_F64 ? maxspeed_launch_t<RPT<double>>(p, lay, q, out, s)           \
                                 : maxspeed_launch_t<RPT<float>>(p, lay, q, out, s);           \
    }                                                                                          \
    }
