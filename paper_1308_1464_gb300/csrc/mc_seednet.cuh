// mc_seednet.cuh -- device layout of the pressure-seed network and the
// per-warp BF16 inference shared by the exact solver and the trainer.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/manyclaw.h"
#include "mc_mma.cuh"

namespace mc {

// offsets in the FP32 parameter vector (see manyclaw.h)
constexpr int P_W1 = 0, P_B1 = 1024, P_W2 = 1088, P_B2 = 5184, P_W3 = 5248, P_B3 = 5312;
constexpr int P_MU = MC_MLP_NWEIGHT, P_SIG = MC_MLP_NWEIGHT + 10;
static_assert(P_B3 + 1 == MC_MLP_NWEIGHT, "parameter layout");
constexpr int NH = 64;
// padded shared/global pitches (BF16 elements) that keep fragment loads
// free of bank conflicts: row r starts at bank 12 r (W1P) or 4 r (W2P, XP2)
constexpr int W1P = 24, W2P = 72, XP = 24;

// Device-resident network: master FP32 parameters, BF16 copies in the
// layouts the mma fragments read, and the optimiser state.
// CTAs of one training launch at most (their partial gradients live in MlpDev)
constexpr int TRAIN_MAX_CTAS = 256;

struct MlpDev {
    float params[MC_MLP_NPARAM];
    __nv_bfloat16 w1t[NH * W1P];   // [out][in]: W1 transposed, 16 inputs used
    __nv_bfloat16 w2t[NH * W2P];   // [out][in]: W2 transposed
    __nv_bfloat16 w2[NH * W2P];    // [in][out]: W2 as stored (for back-propagation)
    float w3r[NH];                  // W3 rounded to BF16, as float
    float grad[MC_MLP_NWEIGHT];
    float adam_m[MC_MLP_NWEIGHT];
    float adam_v[MC_MLP_NWEIGHT];
    double loss_sum;      // sum of squared residuals of the last gradient
    double loss_epoch;    // ... accumulated over an epoch by the optimiser
    int adam_t;
    float gnorm_mean;     // running mean of the clipped gradient norms (0: none yet)
    float gscale;         // factor the optimiser applies to the current gradient
    // per-CTA partial gradients and losses of one training launch, summed in
    // CTA order into grad and loss_sum (deterministic: no float atomics)
    float gpart[TRAIN_MAX_CTAS * MC_MLP_NWEIGHT];
    double lpart[TRAIN_MAX_CTAS];
};

// Rebuilds the BF16 weight copies from the FP32 parameters (mc_exact.cu).
cudaError_t mlp_pack(MlpDev* d, cudaStream_t s);

}  // namespace mc

struct mc_mlp {
    mc::MlpDev* dev;
};

namespace mc {

// Shared-memory copy used by inference.
struct MlpShared {
    __nv_bfloat16 w1t[NH * W1P];
    __nv_bfloat16 w2t[NH * W2P];
    float b1[NH], b2[NH], w3r[NH];
    float mu[10], sig[10];
    float b3;
};

__device__ __forceinline__ void mlp_load_shared(const MlpDev* d, MlpShared* s)
{
    const uint32_t* src1 = reinterpret_cast<const uint32_t*>(d->w1t);
    uint32_t* dst1 = reinterpret_cast<uint32_t*>(s->w1t);
    for (int k = threadIdx.x; k < NH * W1P / 2; k += blockDim.x) dst1[k] = src1[k];
    const uint32_t* src2 = reinterpret_cast<const uint32_t*>(d->w2t);
    uint32_t* dst2 = reinterpret_cast<uint32_t*>(s->w2t);
    for (int k = threadIdx.x; k < NH * W2P / 2; k += blockDim.x) dst2[k] = src2[k];
    for (int k = threadIdx.x; k < NH; k += blockDim.x) {
        s->b1[k] = d->params[P_B1 + k];
        s->b2[k] = d->params[P_B2 + k];
        s->w3r[k] = d->w3r[k];
    }
    for (int k = threadIdx.x; k < 10; k += blockDim.x) {
        s->mu[k] = d->params[P_MU + k];
        s->sig[k] = d->params[P_SIG + k];
    }
    if (threadIdx.x == 0) s->b3 = d->params[P_B3];
}

// Evaluates the network on the 32 rows of the warp: row `lane` holds this
// lane's 16 standardised inputs (10 used).  xs is the warp's [32][XP] BF16
// scratch tile, outs its 32-float scratch.  Every lane must call it.
__device__ __forceinline__ float mlp_infer_warp(const MlpShared& s, const float (&x)[10],
                                                __nv_bfloat16* xs, float* outs)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int k = 0; k < 16; k++) xs[lane * XP + k] = __float2bfloat16_rn(k < 10 ? x[k] : 0.0f);
    __syncwarp();
#pragma unroll 1
    for (int mt = 0; mt < 2; mt++) {
        const int r0 = mt * 16 + g;
        uint32_t a[4];
        a[0] = *reinterpret_cast<const uint32_t*>(&xs[r0 * XP + 2 * t]);
        a[1] = *reinterpret_cast<const uint32_t*>(&xs[(r0 + 8) * XP + 2 * t]);
        a[2] = *reinterpret_cast<const uint32_t*>(&xs[r0 * XP + 2 * t + 8]);
        a[3] = *reinterpret_cast<const uint32_t*>(&xs[(r0 + 8) * XP + 2 * t + 8]);
        // layer 1 -> A fragments of layer 2
        uint32_t a2[4][4];
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            const __nv_bfloat16* wb = &s.w1t[(nt * 8 + g) * W1P + 2 * t];
            mma_bf16_16816(c, a, *reinterpret_cast<const uint32_t*>(wb),
                           *reinterpret_cast<const uint32_t*>(wb + 8));
            const float bb0 = s.b1[nt * 8 + 2 * t], bb1 = s.b1[nt * 8 + 2 * t + 1];
            const uint32_t lo = pack_bf16x2(fmaxf(c[0] + bb0, 0.f), fmaxf(c[1] + bb1, 0.f));
            const uint32_t hi = pack_bf16x2(fmaxf(c[2] + bb0, 0.f), fmaxf(c[3] + bb1, 0.f));
            a2[nt >> 1][(nt & 1) * 2 + 0] = lo;
            a2[nt >> 1][(nt & 1) * 2 + 1] = hi;
        }
        // layer 2 and the 64 -> 1 output on the CUDA cores
        float og = 0.f, og8 = 0.f;
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kb = 0; kb < 4; kb++) {
                const __nv_bfloat16* wb = &s.w2t[(nt * 8 + g) * W2P + kb * 16 + 2 * t];
                mma_bf16_16816(c, a2[kb], *reinterpret_cast<const uint32_t*>(wb),
                               *reinterpret_cast<const uint32_t*>(wb + 8));
            }
            const int n0 = nt * 8 + 2 * t;
            const float bb0 = s.b2[n0], bb1 = s.b2[n0 + 1];
            const float w0 = s.w3r[n0], w1 = s.w3r[n0 + 1];
            og += bf16_round(fmaxf(c[0] + bb0, 0.f)) * w0 + bf16_round(fmaxf(c[1] + bb1, 0.f)) * w1;
            og8 += bf16_round(fmaxf(c[2] + bb0, 0.f)) * w0 + bf16_round(fmaxf(c[3] + bb1, 0.f)) * w1;
        }
        og += __shfl_xor_sync(0xffffffffu, og, 1);
        og += __shfl_xor_sync(0xffffffffu, og, 2);
        og8 += __shfl_xor_sync(0xffffffffu, og8, 1);
        og8 += __shfl_xor_sync(0xffffffffu, og8, 2);
        if (t == 0) {
            outs[r0] = og + s.b3;
            outs[r0 + 8] = og8 + s.b3;
        }
    }
    __syncwarp();
    const float o = outs[lane];
    __syncwarp();
    return o;
}

}  // namespace mc
