// mc_mma.cuh -- warp-level BF16 tensor-core helpers for the seed network.
//
// The network is tiny (10 -> 64 -> 64 -> 1) and is evaluated per warp on
// the 32 interfaces the warp is solving, inside the FP64 Newton kernel, so
// the warp-synchronous mma.sync.m16n8k16 (BF16 operands, FP32 accumulate)
// is the instruction that fits: one warp, 32 rows, weights in shared memory.
//
// Fragment layout of mma.m16n8k16 (PTX ISA, "Matrix Fragments for mma.m16n8k16"),
// with g = lane / 4 and t = lane % 4:
//   A (16 x 16, row major): a0 = A[g][2t..2t+1], a1 = A[g+8][2t..], a2 = A[g][2t+8..],
//                           a3 = A[g+8][2t+8..]          (each a BF16 pair)
//   B (16 x 8, "col major"): b0 = B[2t..2t+1][g], b1 = B[2t+8..2t+9][g]
//   C (16 x 8, FP32):        c0, c1 = C[g][2t], C[g][2t+1]; c2, c3 = C[g+8][2t], C[g+8][2t+1]
// so the C fragments of two adjacent n-tiles form the A fragment of one
// 16-wide k-block of the next layer without leaving registers.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace mc {

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

__device__ __forceinline__ float bf16_round(float x)
{
    return __bfloat162float(__float2bfloat16_rn(x));
}

__device__ __forceinline__ void mma_bf16_16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                               uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

}  // namespace mc
