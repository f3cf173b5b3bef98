// mc_noalloc.cu -- mc_step_noalloc: one unsplit step that allocates no
// device memory.
//
// Some callers cannot call cudaMalloc: plug-ins whose host hands them a fixed
// device-memory budget and owns every allocation, and latency-critical loops
// that must not risk the implicit device synchronisation that allocating and
// freeing can cause.  mc_step needs a
// context (mc_create allocates its device scratch), so this entry point runs
// the same ghost fill and fused step with their scratch -- the running
// maximum of the edge speeds, the device status word and the tensor map the
// TMA reads -- in a file-scope device array instead.  Every call shares that
// array: calls that overlap on the GPU (other streams, other host threads)
// race on it.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>
#include <string.h>

#include <mutex>

#include "mc_device.cuh"
#include "mc_internal.h"
#include "mc_tile.h"

namespace mc {
namespace {

// Scratch of one call: the running speed maximum, the status word, the FP64
// guard's queue counters (FP32 shallow water and Euler) and the tensor map of
// q_in (which the TMA reads from device memory) -- 192 bytes,
// inside an array of NOALLOC_SCRATCH_BYTES that every device loading the
// library keeps until the process exits.
constexpr size_t NOALLOC_SCRATCH_BYTES = 256;
struct NoallocScratch {
    unsigned long long smax_bits;
    int status;
    unsigned guard_queue[2];   // count and done of the FP64 guard's queue (no task list)
    int pad[11];
    CUtensorMap map;   // 64-byte aligned
};
static_assert(offsetof(NoallocScratch, map) % 64 == 0, "tensor map alignment");
static_assert(sizeof(NoallocScratch) <= NOALLOC_SCRATCH_BYTES, "scratch record too large");

__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Per-device set-up, done by the first call on each device (with that device
// current): the device address of the scratch array and the dynamic
// shared-memory limits of every solver's fused kernels in both precisions
// (several need more than the 48 KB default).  The host symbol
// g_noalloc_scratch is only a host-side stand-in; kernels must be given the
// address obtained here.  A set-up that fails is not remembered: the next
// call tries again.
struct DeviceSetup {
    bool done = false;
    NoallocScratch* scratch = nullptr;
};
DeviceSetup g_setup[MAX_DEVICES];
std::mutex g_setup_mutex;
std::once_flag g_encode_once;
EncodeTiledFn g_encode = nullptr;

cudaError_t setup_device(int dev, NoallocScratch** out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup& s = g_setup[dev];
    if (!s.done) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        for (int dtype = MC_F32; e == cudaSuccess && dtype <= MC_F64; dtype++) {
            cudaError_t (*prep[])(int) = {sweep_prepare_acoustics, sweep_prepare_swe,
                                          sweep_prepare_euler, sweep_prepare_advection,
                                          sweep_prepare_acoustics_var, sweep_prepare_euler_godunov};
            for (auto f : prep)
                if (e == cudaSuccess) e = f(dtype);
        }
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return e;
        }
        s.scratch = static_cast<NoallocScratch*>(p);
        s.done = true;
    }
    *out = s.scratch;
    return cudaSuccess;
}

// Starts a call: clears the speed maximum and the status word left by the
// previous call and stores this call's tensor map.  The map travels as a
// kernel argument (copied at launch), so no host buffer has to outlive the
// call.
__global__ void noalloc_begin_kernel(NoallocScratch* s, const CUtensorMap map)
{
    const int t = threadIdx.x;
    const uint64_t* src = reinterpret_cast<const uint64_t*>(&map);
    uint64_t* dst = reinterpret_cast<uint64_t*>(&s->map);
    if (t < int(sizeof(CUtensorMap) / 8)) dst[t] = src[t];
    if (t == 0) {
        s->smax_bits = 0ull;
        s->status = 0;
        s->guard_queue[0] = s->guard_queue[1] = 0u;
    }
}

}  // namespace
}  // namespace mc

using namespace mc;

extern "C" mc_status mc_step_noalloc(const mc_problem* p, void* q_in, void* q_out, double dt,
                                     double* smax_out, void* stream)
{
    mc_layout lay;
    mc_status st = mc_layout_of(p, &lay);
    if (st != MC_OK) return st;
    if (!q_in || !q_out) return set_error(MC_EINVAL, "NULL state pointer");
    if (q_in == q_out) return set_error(MC_EINVAL, "q_in and q_out must differ");
    if (reinterpret_cast<uintptr_t>(q_in) % 16 || reinterpret_cast<uintptr_t>(q_out) % 16)
        return set_error(MC_EINVAL, "state pointers must be 16-byte aligned");
    if (!(dt >= 0.0) || !isfinite(dt)) return set_error(MC_EINVAL, "dt must be finite and >= 0");
    // The scratch a call needs does not grow with the grid (the static_assert
    // above keeps the record inside the array), so every grid that
    // mc_layout_of accepts fits; larger grids were refused there.
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= MAX_DEVICES) return set_error(MC_EINVAL, "device %d out of range", dev);
    NoallocScratch* scratch = nullptr;
    e = setup_device(dev, &scratch);
    if (e != cudaSuccess) return cuda_error(e, "per-device set-up (cudaGetSymbolAddress)");
    std::call_once(g_encode_once, []() {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<EncodeTiledFn>(fn);
    });
    if (!g_encode) return set_error(MC_ECUDA, "driver entry point cuTensorMapEncodeTiled unavailable");

    // tensor map of q_in, encoded on the host and stored into the array
    const int es = (int)lay.elem_bytes;
    cuuint64_t dims[3] = {(cuuint64_t)lay.ld_x, (cuuint64_t)(p->my + 4), (cuuint64_t)lay.meqn};
    cuuint64_t strides[2] = {(cuuint64_t)(lay.ld_x * es), (cuuint64_t)(lay.ld_field * es)};
    cuuint32_t box[3] = {(cuuint32_t)box_w(es), (cuuint32_t)stage_rows(es), (cuuint32_t)lay.meqn};
    cuuint32_t estr[3] = {1, 1, 1};
    CUtensorMap map;
    CUresult r = g_encode(&map,
                          es == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                          3, q_in, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(MC_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the array keeps the previous call's contents: the maximum and the
    // status word must start from zero; the map is rewritten every call
    noalloc_begin_kernel<<<1, 32, 0, s>>>(scratch, map);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = bc_launch(*p, lay, q_in, q_in, nullptr, s);
    if (e != cudaSuccess) return cuda_error(e, "ghost fill");
    const int rows = DEFAULT_TILE_ROWS;
    SweepLaunch L{*p, lay, &scratch->map, &scratch->map, q_in, q_out, nullptr, nullptr, dt,
                  &scratch->smax_bits, &scratch->status, rows, 0, s};
    // the FP64 guard recomputes every task of a step that queued one (the
    // array has no room for a task list)
    L.gq = scratch->guard_queue;
    switch (p->solver) {
    case MC_ACOUSTICS: e = sweep_launch_acoustics(L); break;
    case MC_SWE_ROE: e = sweep_launch_swe(L); break;
    case MC_ADVECTION: e = sweep_launch_advection(L); break;
    case MC_ACOUSTICS_VAR: e = sweep_launch_acoustics_var(L); break;
    case MC_EULER_GODUNOV: e = sweep_launch_euler_godunov(L); break;
    default: e = sweep_launch_euler(L); break;
    }
    if (e != cudaSuccess) return cuda_error(e, "sweep launch");
    if (smax_out) {
        NoallocScratch h;
        e = cudaMemcpyAsync(&h, scratch, offsetof(NoallocScratch, map), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_error(e, "reading the step's scratch");
        memcpy(smax_out, &h.smax_bits, sizeof(double));
        if (h.status & ST_BADARG)
            return set_error(MC_EINVAL, "the fused step found a misaligned tensor map or box");
        if (h.status & ST_TIMEOUT) return set_error(MC_ETIMEOUT, "a bounded device wait gave up");
        if (h.status & ST_NONPHYS)
            return set_error(MC_ENONPHYS, "non-physical state (depth/density <= 0 or NaN) met");
    }
    return MC_OK;
}
