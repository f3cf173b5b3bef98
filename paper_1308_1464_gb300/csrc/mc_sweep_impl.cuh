// mc_sweep_impl.cuh -- launch code of the fused step for one Riemann solver;
// included once per solver translation unit.
#pragma once

#include "mc_batch.cuh"
#include "mc_internal.h"
#include "mc_multi.cuh"
#include "mc_sweep.cuh"

namespace mc {

// dynamic shared memory the seed network adds to the fused step: its shared
// copy, then per warp the [32][XP] BF16 input tile and 32 output floats
inline int seednet_smem_bytes()
{
    return int(sizeof(MlpShared)) + SWEEP_WARPS * 32 * XP * 2 + SWEEP_WARPS * 32 * 4;
}

// the compile-time scheme of a problem's fused step: MODE_FAST for MC,
// second order, transverse option 1; MODE_TRANS2 for second order with
// transverse option 2; MODE_GENERAL otherwise
inline int scheme_mode(const mc_problem& p)
{
    if (p.limiter == MC_LIM_MC && p.order == 2 && p.transverse == 1) return MODE_FAST;
    if (p.order == 2 && p.transverse == 2) return MODE_TRANS2;
    return MODE_GENERAL;
}

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
    a.split = L.tile_split;
    a.ntasks = ntasks_split(L.prob, L.tile_rows, L.tile_split, &a.nbands, &a.nbig);
    a.smax_bits = L.smax_bits;
    a.status = L.status;
    a.net = RP::SEEDED ? static_cast<const MlpDev*>(L.seed_net) : nullptr;
    a.newton_updates = RP::SEEDED ? L.newton : nullptr;
    a.guard_edges = RP::PAIRED ? L.guard : nullptr;
    a.gq = RP::PAIRED ? static_cast<GuardQueue*>(L.gq) : nullptr;
    a.gq_tasks = RP::PAIRED ? L.gq_tasks : nullptr;
    // the guard kernel applies the time-step rule only where it runs
    a.dt_state = nullptr;
    if constexpr (RP::PAIRED) {
        if (a.gq && a.rp.guard_on()) a.dt_state = L.dt_state;
    }
    a.cfl_desired = L.cfl_desired;
    a.cfl_max = L.cfl_max;
    if (L.dt_folded) *L.dt_folded = a.dt_state != nullptr;

    const int smem = sweep_smem_bytes(sizeof(T), RP::NPLANE) + (a.net ? seednet_smem_bytes() : 0);
    // a grid with fewer tasks than SWEEP_WARPS per SM gets smaller CTAs, so
    // that its warps land on separate SMs instead of sharing a few
    int wpb = SWEEP_WARPS;
    if (L.sms > 0 && a.ntasks < L.sms * SWEEP_WARPS) {
        wpb = (a.ntasks + L.sms - 1) / L.sms;
        if (wpb < 1) wpb = 1;
    }
    int blocks = (a.ntasks + wpb - 1) / wpb;
    if (L.max_blocks > 0 && blocks > L.max_blocks) blocks = L.max_blocks;
    const int mode = scheme_mode(L.prob);
    switch (mode) {
    case MODE_FAST:
        ctu_sweep_kernel<RP, MODE_FAST><<<blocks, wpb * 32, smem, L.stream>>>(L.map_a, L.map_b, a);
        break;
    case MODE_TRANS2:
        ctu_sweep_kernel<RP, MODE_TRANS2><<<blocks, wpb * 32, smem, L.stream>>>(L.map_a, L.map_b, a);
        break;
    default:
        ctu_sweep_kernel<RP, MODE_GENERAL><<<blocks, wpb * 32, smem, L.stream>>>(L.map_a, L.map_b, a);
    }
    if constexpr (RP::PAIRED) {
        // the FP64 guard's recompute of the tasks the step queued
        if (a.gq && a.rp.guard_on()) {
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            int gblocks = (a.ntasks + SWEEP_WARPS - 1) / SWEEP_WARPS;
            const int cap = 2 * (L.sms > 0 ? L.sms : 152);
            if (gblocks > cap) gblocks = cap;
            switch (mode) {
            case MODE_FAST:
                ctu_guard_kernel<RP, MODE_FAST><<<gblocks, SWEEP_WARPS * 32, smem, L.stream>>>(L.map_a, L.map_b, a);
                break;
            case MODE_TRANS2:
                ctu_guard_kernel<RP, MODE_TRANS2><<<gblocks, SWEEP_WARPS * 32, smem, L.stream>>>(L.map_a, L.map_b, a);
                break;
            default:
                ctu_guard_kernel<RP, MODE_GENERAL><<<gblocks, SWEEP_WARPS * 32, smem, L.stream>>>(L.map_a, L.map_b, a);
            }
        }
    }
    return cudaGetLastError();
}

// Raises the kernel's dynamic shared-memory limit; called once per context
// (outside any stream capture) before the first launch.
template <class RP>
cudaError_t sweep_prepare_t()
{
    using T = typename RP::real;
    const int smem = sweep_smem_bytes(sizeof(T), RP::NPLANE) + (RP::SEEDED ? seednet_smem_bytes() : 0);
    cudaError_t e = cudaFuncSetAttribute(ctu_sweep_kernel<RP, MODE_FAST>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ctu_sweep_kernel<RP, MODE_TRANS2>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ctu_sweep_kernel<RP, MODE_GENERAL>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if constexpr (RP::PAIRED) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(ctu_guard_kernel<RP, MODE_FAST>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(ctu_guard_kernel<RP, MODE_TRANS2>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(ctu_guard_kernel<RP, MODE_GENERAL>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    }
    return e;
}

template <class RP>
cudaError_t maxspeed_launch_t(const mc_problem& p, const mc_layout& lay, const void* q,
                              unsigned long long* out, cudaStream_t s)
{
    using T = typename RP::real;
    RP rp;
    rp.setup(p.param, p.efix);
    int blocks = (p.my + 7) / 8;   // 8 warps of 256 threads, one row each
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    max_cell_speed_kernel<RP><<<blocks, 256, 0, s>>>(rp, static_cast<const T*>(q), p.mx, p.my,
                                                      lay.ld_x, lay.ld_field, lay.x_offset, p.dx,
                                                      p.dy, out);
    return cudaGetLastError();
}

template <class RP>
BatchArgs<RP> batch_args(const BatchLaunch& L)
{
    BatchArgs<RP> a;
    a.rp.setup(L.proto.param, L.proto.efix);
    a.patches = L.patches;
    a.maps = L.maps;
    a.prefix = L.prefix;
    a.npatch = L.npatch;
    a.nsteps = L.nsteps;
    a.step0 = L.step0;
    a.nsteps_all = L.nsteps_all > 0 ? L.nsteps_all : L.nsteps;
    a.tasks_per_step = L.tasks_per_step;
    a.x_offset = L.x_offset;
    a.cfl = L.cfl;
    a.limiter = L.proto.limiter;
    a.order = L.proto.order;
    a.transverse = L.proto.transverse;
    a.smax = L.smax;
    a.dt_used = L.dt_used;
    a.done = L.done;
    a.next_item = L.next_item;
    a.status = L.status;
    return a;
}

template <class RP>
cudaError_t batch_launch_t(const BatchLaunch& L)
{
    using T = typename RP::real;
    constexpr int smem = sweep_smem_bytes(sizeof(T), RP::NPLANE);
    switch (scheme_mode(L.proto)) {
    case MODE_FAST:
        batch_sweep_kernel<RP, MODE_FAST><<<L.blocks, SWEEP_WARPS * 32, smem, L.stream>>>(batch_args<RP>(L));
        break;
    case MODE_TRANS2:
        batch_sweep_kernel<RP, MODE_TRANS2><<<L.blocks, SWEEP_WARPS * 32, smem, L.stream>>>(batch_args<RP>(L));
        break;
    default:
        batch_sweep_kernel<RP, MODE_GENERAL><<<L.blocks, SWEEP_WARPS * 32, smem, L.stream>>>(batch_args<RP>(L));
    }
    return cudaGetLastError();
}

template <class RP>
cudaError_t batch_init_t(const BatchLaunch& L)
{
    RP rp;
    rp.setup(L.proto.param, L.proto.efix);
    // four blocks per patch (a patch has at most a few hundred rows)
    const dim3 grid(4, (unsigned)(L.npatch < 1 ? 1 : L.npatch < 65535 ? L.npatch : 65535));
    batch_init_kernel<RP><<<grid, 256, 0, L.stream>>>(rp, L.patches, L.npatch, L.x_offset,
                                                     (L.nsteps_all > 0 ? L.nsteps_all : L.nsteps) + 1,
                                                     L.smax);
    return cudaGetLastError();
}

// CTAs of the fused step's kernel (the problem's compiled scheme) resident
// on one SM; the kernel's shared-memory limit must be raised already
template <class RP>
cudaError_t sweep_occupancy_t(const mc_problem& p, int* ctas)
{
    using T = typename RP::real;
    const int smem = sweep_smem_bytes(sizeof(T), RP::NPLANE) + (RP::SEEDED ? seednet_smem_bytes() : 0);
    switch (scheme_mode(p)) {
    case MODE_FAST:
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, ctu_sweep_kernel<RP, MODE_FAST>,
                                                             SWEEP_WARPS * 32, smem);
    case MODE_TRANS2:
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, ctu_sweep_kernel<RP, MODE_TRANS2>,
                                                             SWEEP_WARPS * 32, smem);
    default:
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, ctu_sweep_kernel<RP, MODE_GENERAL>,
                                                             SWEEP_WARPS * 32, smem);
    }
}

template <class RP>
cudaError_t batch_occupancy_t(int* ctas)
{
    using T = typename RP::real;
    constexpr int smem = sweep_smem_bytes(sizeof(T), RP::NPLANE);
    cudaError_t e = cudaFuncSetAttribute(batch_sweep_kernel<RP, MODE_FAST>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batch_sweep_kernel<RP, MODE_TRANS2>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batch_sweep_kernel<RP, MODE_GENERAL>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, batch_sweep_kernel<RP, MODE_FAST>,
                                                         SWEEP_WARPS * 32, smem);
}

template <class RP>
cudaError_t multi_launch_t(const MultiLaunch& L)
{
    using T = typename RP::real;
    MultiArgs<RP> a;
    a.rp.setup(L.prob.param, L.prob.efix);
    a.grids = static_cast<const MultiGrid*>(L.grids);
    a.maps = L.maps;
    a.prefix = L.prefix;
    a.ngrid = L.ngrid;
    a.cur = L.cur;
    a.total = L.total;
    a.x_offset = L.x_offset;
    a.nux = L.nux;
    a.nuy = L.nuy;
    a.limiter = L.prob.limiter;
    a.order = L.prob.order;
    a.transverse = L.prob.transverse;
    a.status = L.status;
    constexpr int smem = sweep_smem_bytes(sizeof(T), RP::NPLANE);
    long long blocks = (L.total + SWEEP_WARPS - 1) / SWEEP_WARPS;
    if (blocks < 1) blocks = 1;
    cudaError_t e;
    switch (scheme_mode(L.prob)) {
    case MODE_FAST:
        e = cudaFuncSetAttribute(multi_sweep_kernel<RP, MODE_FAST>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            multi_sweep_kernel<RP, MODE_FAST><<<(unsigned)blocks, SWEEP_WARPS * 32, smem, L.stream>>>(a);
        break;
    case MODE_TRANS2:
        e = cudaFuncSetAttribute(multi_sweep_kernel<RP, MODE_TRANS2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            multi_sweep_kernel<RP, MODE_TRANS2><<<(unsigned)blocks, SWEEP_WARPS * 32, smem, L.stream>>>(a);
        break;
    default:
        e = cudaFuncSetAttribute(multi_sweep_kernel<RP, MODE_GENERAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            multi_sweep_kernel<RP, MODE_GENERAL><<<(unsigned)blocks, SWEEP_WARPS * 32, smem, L.stream>>>(a);
    }
    return e == cudaSuccess ? cudaGetLastError() : e;
}

}  // namespace mc

#define MC_DEFINE_SOLVER_LAUNCHERS(NAME, RPT)                                                  \
    namespace mc {                                                                             \
    cudaError_t multi_launch_##NAME(const MultiLaunch& L)                                      \
    {                                                                                          \
        return L.prob.dtype == MC_F64 ? multi_launch_t<RPT<double>>(L)                         \
                                      : multi_launch_t<RPT<float>>(L);                         \
    }                                                                                          \
    cudaError_t sweep_launch_##NAME(const SweepLaunch& L)                                      \
    {                                                                                          \
        return L.prob.dtype == MC_F64 ? sweep_launch_t<RPT<double>>(L)                         \
                                      : sweep_launch_t<RPT<float>>(L);                         \
    }                                                                                          \
    cudaError_t sweep_prepare_##NAME(int dtype)                                                \
    {                                                                                          \
        return dtype == MC_F64 ? sweep_prepare_t<RPT<double>>() : sweep_prepare_t<RPT<float>>(); \
    }                                                                                          \
    cudaError_t sweep_occupancy_##NAME(const mc_problem& p, int* ctas)                         \
    {                                                                                          \
        return p.dtype == MC_F64 ? sweep_occupancy_t<RPT<double>>(p, ctas)                     \
                                 : sweep_occupancy_t<RPT<float>>(p, ctas);                     \
    }                                                                                          \
    cudaError_t batch_launch_##NAME(const BatchLaunch& L)                                      \
    {                                                                                          \
        return L.proto.dtype == MC_F64 ? batch_launch_t<RPT<double>>(L)                        \
                                       : batch_launch_t<RPT<float>>(L);                        \
    }                                                                                          \
    cudaError_t batch_init_##NAME(const BatchLaunch& L)                                        \
    {                                                                                          \
        return L.proto.dtype == MC_F64 ? batch_init_t<RPT<double>>(L)                          \
                                       : batch_init_t<RPT<float>>(L);                          \
    }                                                                                          \
    cudaError_t batch_occupancy_##NAME(int dtype, int* ctas)                                   \
    {                                                                                          \
        return dtype == MC_F64 ? batch_occupancy_t<RPT<double>>(ctas)                          \
                               : batch_occupancy_t<RPT<float>>(ctas);                          \
    }                                                                                          \
    cudaError_t maxspeed_launch_##NAME(const mc_problem& p, const mc_layout& lay,              \
                                       const void* q, unsigned long long* out, cudaStream_t s) \
    {                                                                                          \
        return p.dtype == MC_F64 ? maxspeed_launch_t<RPT<double>>(p, lay, q, out, s)           \
                                 : maxspeed_launch_t<RPT<float>>(p, lay, q, out, s);           \
    }                                                                                          \
    }
