// mc_mlp.cu -- forward, back-propagation and Adam training of the pressure
// seed network on the tensor cores (mc_mlp_forward, mc_mlp_grad,
// mc_mlp_train).
//
// One warp takes 16 rows at a time through the whole network and back:
//   forward   H1 = relu(X W1 + b1), H2 = relu(H1 W2 + b2), out = H2 W3 + b3
//   backward  dout = 2 (out - y) / B
//             D2 = dout W3^T . [H2 > 0]          gW3 += H2^T dout, gb3 += sum dout
//             gW2 += H1^T D2,  gb2 += sum D2
//             D1 = (D2 W2^T) . [H1 > 0]           gb1 += sum D1
//             gW1 += X^T D1
// Every product of activations, weights or activation gradients takes BF16
// operands with FP32 accumulation (mma.sync.m16n8k16); the 64 -> 1 layer and
// the bias sums stay on the CUDA cores in FP32.  The transposed operands of
// the weight-gradient products (H1^T, X^T as A; D2, D1 as B) are staged in
// shared memory, transposed, so that every fragment is one 32-bit load.
// Gradients accumulate per warp in shared memory (contributions of several
// lanes to one weight are first summed by shuffles in a fixed order), the
// warps' sums are added in warp order into a per-CTA partial, and a second
// kernel adds the partials in CTA order: no float atomics, so a training run
// is bitwise reproducible.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <vector>

#include "mc_internal.h"
#include "mc_seednet.cuh"

namespace mc {

constexpr int TW = 4;       // warps per CTA
constexpr int BP = 24;      // pitch of the transposed [feature][row] tiles (16 rows used)

struct TrainShared {
    __nv_bfloat16 w1t[NH * W1P];
    __nv_bfloat16 w2t[NH * W2P];
    __nv_bfloat16 w2[NH * W2P];
    float b1[NH], b2[NH], w3r[NH];
    float mu[10], sig[10];
    float b3;
    float g[TW][MC_MLP_NWEIGHT];              // per-warp gradients
    float loss[TW];
    struct Warp {
        __nv_bfloat16 xs[16 * XP];            // X, row major (A of layer 1)
        __nv_bfloat16 xT[16 * BP];            // X^T  [feature][row]
        __nv_bfloat16 h1T[NH * BP];           // H1^T [unit][row]
        __nv_bfloat16 d2T[NH * BP];           // D2^T [unit][row]
        __nv_bfloat16 d1T[NH * BP];           // D1^T [unit][row]
        float y[16];
        float valid[16];
    } w[TW];
};

struct TrainArgs {
    MlpDev* net;
    long long n;           // rows in the dataset
    long long rows;        // rows of this call (a batch)
    long long first;       // position of the batch in the epoch's order
    long long perm_a, perm_b;   // order: row(k) = (a k + b) mod n
    const float* feat;     // n x 10 raw features
    const float* target;   // n
    float inv_batch;       // 1 / rows
    int backward;          // 0: forward only (out), 1: gradients
    float* out;            // forward output per row of this call (nullable)
};

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p)
{
    return *reinterpret_cast<const uint32_t*>(p);
}

__global__ void __launch_bounds__(TW * 32) mlp_train_kernel(const TrainArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainShared& S = *reinterpret_cast<TrainShared*>(smem_raw);
    const MlpDev* d = a.net;
    // weights into shared memory, CTA gradient to zero
    {
        const uint32_t* s1 = reinterpret_cast<const uint32_t*>(d->w1t);
        uint32_t* t1 = reinterpret_cast<uint32_t*>(S.w1t);
        for (int k = threadIdx.x; k < NH * W1P / 2; k += blockDim.x) t1[k] = s1[k];
        const uint32_t* s2 = reinterpret_cast<const uint32_t*>(d->w2t);
        uint32_t* t2 = reinterpret_cast<uint32_t*>(S.w2t);
        const uint32_t* s3 = reinterpret_cast<const uint32_t*>(d->w2);
        uint32_t* t3 = reinterpret_cast<uint32_t*>(S.w2);
        for (int k = threadIdx.x; k < NH * W2P / 2; k += blockDim.x) {
            t2[k] = s2[k];
            t3[k] = s3[k];
        }
        for (int k = threadIdx.x; k < NH; k += blockDim.x) {
            S.b1[k] = d->params[P_B1 + k];
            S.b2[k] = d->params[P_B2 + k];
            S.w3r[k] = d->w3r[k];
        }
        for (int k = threadIdx.x; k < 10; k += blockDim.x) {
            S.mu[k] = d->params[P_MU + k];
            S.sig[k] = d->params[P_SIG + k];
        }
        float* g0 = &S.g[0][0];
        for (int k = threadIdx.x; k < TW * MC_MLP_NWEIGHT; k += blockDim.x) g0[k] = 0.f;
        if (threadIdx.x < TW) S.loss[threadIdx.x] = 0.f;
        if (threadIdx.x == 0) S.b3 = d->params[P_B3];
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    TrainShared::Warp& W = S.w[warp];
    float* G = S.g[warp];
    // sum over the eight lanes of one t (lanes t, t + 4, ..., t + 28), fixed order
    auto sum_g = [](float v) {
        v += __shfl_xor_sync(0xffffffffu, v, 4);
        v += __shfl_xor_sync(0xffffffffu, v, 8);
        v += __shfl_xor_sync(0xffffffffu, v, 16);
        return v;
    };
    const long long nchunk = (a.rows + 15) / 16;
    for (long long ch = (long long)blockIdx.x * TW + warp; ch < nchunk;
         ch += (long long)gridDim.x * TW) {
        // ---- stage 16 rows: standardised inputs (BF16), targets, validity
        if (lane < 16) {
            const long long k = ch * 16 + lane;
            float x[10], y = 0.f, ok = 0.f;
            if (k < a.rows) {
                const long long row = (a.perm_a * ((a.first + k) % a.n) + a.perm_b) % a.n;
                bool fin = true;
#pragma unroll
                for (int f = 0; f < 10; f++) {
                    x[f] = a.feat[row * 10 + f];
                    fin = fin && isfinite(x[f]);
                }
                y = a.target ? a.target[row] : 0.f;
                ok = (fin && isfinite(y)) ? 1.f : 0.f;
            }
#pragma unroll
            for (int f = 0; f < 10; f++) {
                const float v = ok > 0.f ? (x[f] - S.mu[f]) / S.sig[f] : 0.f;
                const __nv_bfloat16 b = __float2bfloat16_rn(v);
                W.xs[lane * XP + f] = b;
                W.xT[f * BP + lane] = b;
            }
#pragma unroll
            for (int f = 10; f < 16; f++) {
                W.xs[lane * XP + f] = __float2bfloat16_rn(0.f);
                W.xT[f * BP + lane] = __float2bfloat16_rn(0.f);
            }
            W.y[lane] = ok > 0.f ? y : 0.f;
            W.valid[lane] = ok;
        }
        __syncwarp();

        // ---- forward
        uint32_t ax[4];
        ax[0] = ld_pair(&W.xs[g * XP + 2 * t]);
        ax[1] = ld_pair(&W.xs[(g + 8) * XP + 2 * t]);
        ax[2] = ld_pair(&W.xs[g * XP + 2 * t + 8]);
        ax[3] = ld_pair(&W.xs[(g + 8) * XP + 2 * t + 8]);
        float h1[8][4];
        uint32_t a2[4][4];
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            const __nv_bfloat16* wb = &S.w1t[(nt * 8 + g) * W1P + 2 * t];
            mma_bf16_16816(c, ax, ld_pair(wb), ld_pair(wb + 8));
            const int j0 = nt * 8 + 2 * t;
            h1[nt][0] = bf16_round(fmaxf(c[0] + S.b1[j0], 0.f));
            h1[nt][1] = bf16_round(fmaxf(c[1] + S.b1[j0 + 1], 0.f));
            h1[nt][2] = bf16_round(fmaxf(c[2] + S.b1[j0], 0.f));
            h1[nt][3] = bf16_round(fmaxf(c[3] + S.b1[j0 + 1], 0.f));
            a2[nt >> 1][(nt & 1) * 2 + 0] = pack_bf16x2(h1[nt][0], h1[nt][1]);
            a2[nt >> 1][(nt & 1) * 2 + 1] = pack_bf16x2(h1[nt][2], h1[nt][3]);
            W.h1T[j0 * BP + g] = __float2bfloat16_rn(h1[nt][0]);
            W.h1T[(j0 + 1) * BP + g] = __float2bfloat16_rn(h1[nt][1]);
            W.h1T[j0 * BP + g + 8] = __float2bfloat16_rn(h1[nt][2]);
            W.h1T[(j0 + 1) * BP + g + 8] = __float2bfloat16_rn(h1[nt][3]);
        }
        float h2[8][4];
        float og = 0.f, og8 = 0.f;
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kb = 0; kb < 4; kb++) {
                const __nv_bfloat16* wb = &S.w2t[(nt * 8 + g) * W2P + kb * 16 + 2 * t];
                mma_bf16_16816(c, a2[kb], ld_pair(wb), ld_pair(wb + 8));
            }
            const int k0 = nt * 8 + 2 * t;
            h2[nt][0] = bf16_round(fmaxf(c[0] + S.b2[k0], 0.f));
            h2[nt][1] = bf16_round(fmaxf(c[1] + S.b2[k0 + 1], 0.f));
            h2[nt][2] = bf16_round(fmaxf(c[2] + S.b2[k0], 0.f));
            h2[nt][3] = bf16_round(fmaxf(c[3] + S.b2[k0 + 1], 0.f));
            og += h2[nt][0] * S.w3r[k0] + h2[nt][1] * S.w3r[k0 + 1];
            og8 += h2[nt][2] * S.w3r[k0] + h2[nt][3] * S.w3r[k0 + 1];
        }
        og += __shfl_xor_sync(0xffffffffu, og, 1);
        og += __shfl_xor_sync(0xffffffffu, og, 2);
        og8 += __shfl_xor_sync(0xffffffffu, og8, 1);
        og8 += __shfl_xor_sync(0xffffffffu, og8, 2);
        og += S.b3;
        og8 += S.b3;
        if (!a.backward) {
            if (t == 0 && a.out) {
                const long long k = ch * 16 + g, k8 = k + 8;
                if (k < a.rows) a.out[k] = og;
                if (k8 < a.rows) a.out[k8] = og8;
            }
            __syncwarp();
            continue;
        }

        // ---- backward
        const float vg = W.valid[g], vg8 = W.valid[g + 8];
        const float rg = (og - W.y[g]) * vg, rg8 = (og8 - W.y[g + 8]) * vg8;
        const float dg = 2.f * rg * a.inv_batch, dg8 = 2.f * rg8 * a.inv_batch;
        {
            const float l = sum_g(rg * rg + rg8 * rg8), b = sum_g(dg + dg8);
            if (lane == 0) {
                S.loss[warp] += l;
                G[P_B3] += b;
            }
        }
        float d2[8][4];
        uint32_t ad2[4][4];
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
            const int k0 = nt * 8 + 2 * t;
            const float w0 = S.w3r[k0], w1 = S.w3r[k0 + 1];
            const float gw0 = sum_g(h2[nt][0] * dg + h2[nt][2] * dg8);
            const float gw1 = sum_g(h2[nt][1] * dg + h2[nt][3] * dg8);
            d2[nt][0] = h2[nt][0] > 0.f ? dg * w0 : 0.f;
            d2[nt][1] = h2[nt][1] > 0.f ? dg * w1 : 0.f;
            d2[nt][2] = h2[nt][2] > 0.f ? dg8 * w0 : 0.f;
            d2[nt][3] = h2[nt][3] > 0.f ? dg8 * w1 : 0.f;
            const float gb0 = sum_g(d2[nt][0] + d2[nt][2]), gb1 = sum_g(d2[nt][1] + d2[nt][3]);
            if (g == 0) {
                G[P_W3 + k0] += gw0;
                G[P_W3 + k0 + 1] += gw1;
                G[P_B2 + k0] += gb0;
                G[P_B2 + k0 + 1] += gb1;
            }
            ad2[nt >> 1][(nt & 1) * 2 + 0] = pack_bf16x2(d2[nt][0], d2[nt][1]);
            ad2[nt >> 1][(nt & 1) * 2 + 1] = pack_bf16x2(d2[nt][2], d2[nt][3]);
            W.d2T[k0 * BP + g] = __float2bfloat16_rn(d2[nt][0]);
            W.d2T[(k0 + 1) * BP + g] = __float2bfloat16_rn(d2[nt][1]);
            W.d2T[k0 * BP + g + 8] = __float2bfloat16_rn(d2[nt][2]);
            W.d2T[(k0 + 1) * BP + g + 8] = __float2bfloat16_rn(d2[nt][3]);
        }
        __syncwarp();
        // gW2 += H1^T D2   (M = 64 inputs j, N = 64 outputs k, K = 16 rows)
#pragma unroll 1
        for (int mj = 0; mj < 4; mj++) {
            uint32_t ah[4];
            const int j0 = mj * 16 + g;
            ah[0] = ld_pair(&W.h1T[j0 * BP + 2 * t]);
            ah[1] = ld_pair(&W.h1T[(j0 + 8) * BP + 2 * t]);
            ah[2] = ld_pair(&W.h1T[j0 * BP + 2 * t + 8]);
            ah[3] = ld_pair(&W.h1T[(j0 + 8) * BP + 2 * t + 8]);
#pragma unroll
            for (int nt = 0; nt < 8; nt++) {
                float c[4] = {0.f, 0.f, 0.f, 0.f};
                const __nv_bfloat16* bb = &W.d2T[(nt * 8 + g) * BP + 2 * t];
                mma_bf16_16816(c, ah, ld_pair(bb), ld_pair(bb + 8));
                const int k0 = nt * 8 + 2 * t;
                // each lane owns its four weights of this tile
                G[P_W2 + j0 * NH + k0] += c[0];
                G[P_W2 + j0 * NH + k0 + 1] += c[1];
                G[P_W2 + (j0 + 8) * NH + k0] += c[2];
                G[P_W2 + (j0 + 8) * NH + k0 + 1] += c[3];
            }
        }
        // D1 = (D2 W2^T) . [H1 > 0]
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kb = 0; kb < 4; kb++) {
                const __nv_bfloat16* wb = &S.w2[(nt * 8 + g) * W2P + kb * 16 + 2 * t];
                mma_bf16_16816(c, ad2[kb], ld_pair(wb), ld_pair(wb + 8));
            }
            const int j0 = nt * 8 + 2 * t;
            const float e0 = h1[nt][0] > 0.f ? c[0] : 0.f, e1 = h1[nt][1] > 0.f ? c[1] : 0.f;
            const float e2 = h1[nt][2] > 0.f ? c[2] : 0.f, e3 = h1[nt][3] > 0.f ? c[3] : 0.f;
            {
                const float b0 = sum_g(e0 + e2), b1 = sum_g(e1 + e3);
                if (g == 0) {
                    G[P_B1 + j0] += b0;
                    G[P_B1 + j0 + 1] += b1;
                }
            }
            W.d1T[j0 * BP + g] = __float2bfloat16_rn(e0);
            W.d1T[(j0 + 1) * BP + g] = __float2bfloat16_rn(e1);
            W.d1T[j0 * BP + g + 8] = __float2bfloat16_rn(e2);
            W.d1T[(j0 + 1) * BP + g + 8] = __float2bfloat16_rn(e3);
        }
        __syncwarp();
        // gW1 += X^T D1   (M = 16 inputs, N = 64 units, K = 16 rows)
        {
            uint32_t axt[4];
            axt[0] = ld_pair(&W.xT[g * BP + 2 * t]);
            axt[1] = ld_pair(&W.xT[(g + 8) * BP + 2 * t]);
            axt[2] = ld_pair(&W.xT[g * BP + 2 * t + 8]);
            axt[3] = ld_pair(&W.xT[(g + 8) * BP + 2 * t + 8]);
#pragma unroll
            for (int nt = 0; nt < 8; nt++) {
                float c[4] = {0.f, 0.f, 0.f, 0.f};
                const __nv_bfloat16* bb = &W.d1T[(nt * 8 + g) * BP + 2 * t];
                mma_bf16_16816(c, axt, ld_pair(bb), ld_pair(bb + 8));
                const int j0 = nt * 8 + 2 * t;
                G[P_W1 + g * NH + j0] += c[0];
                G[P_W1 + g * NH + j0 + 1] += c[1];
                G[P_W1 + (g + 8) * NH + j0] += c[2];
                G[P_W1 + (g + 8) * NH + j0 + 1] += c[3];
            }
        }
        __syncwarp();
    }
    if (!a.backward) return;
    __syncthreads();
    // this CTA's partial: the warps' sums in warp order
    float* part = a.net->gpart + (size_t)blockIdx.x * MC_MLP_NWEIGHT;
    for (int k = threadIdx.x; k < MC_MLP_NWEIGHT; k += blockDim.x) {
        float v = S.g[0][k];
#pragma unroll
        for (int w = 1; w < TW; w++) v += S.g[w][k];
        part[k] = v;
    }
    if (threadIdx.x == 0) {
        double l = 0.0;
        for (int w = 0; w < TW; w++) l += double(S.loss[w]);
        a.net->lpart[blockIdx.x] = l;
    }
}

// The gradient and loss of a training launch: its CTAs' partials added in
// CTA order.
__global__ void reduce_grad_kernel(MlpDev* d, int nparts)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < MC_MLP_NWEIGHT;
         k += blockDim.x * gridDim.x) {
        float v = 0.f;
        for (int b = 0; b < nparts; b++) v += d->gpart[(size_t)b * MC_MLP_NWEIGHT + k];
        d->grad[k] = v;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double l = 0.0;
        for (int b = 0; b < nparts; b++) l += d->lpart[b];
        d->loss_sum = l;
    }
}

constexpr int TRAIN_SMEM = (int)sizeof(TrainShared);

__global__ void zero_grad_kernel(MlpDev* d)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < MC_MLP_NWEIGHT;
         k += blockDim.x * gridDim.x)
        d->grad[k] = 0.f;
    if (blockIdx.x == 0 && threadIdx.x == 0) d->loss_sum = 0.0;
}

// Gradient clipping against the running mean of the gradient norms: a step
// whose norm exceeds clip times that mean is scaled down to it, so that a
// minibatch dominated by a few extreme rows (near-vacuum interfaces, whose
// two-rarefaction guess collapses) cannot throw the weights far; the mean
// follows the clipped norms (weight 0.01 per step).  One block.
__global__ void clip_kernel(MlpDev* d, float clip)
{
    __shared__ float part[256];
    float s = 0.f;
    for (int k = threadIdx.x; k < MC_MLP_NWEIGHT; k += blockDim.x) s += d->grad[k] * d->grad[k];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const float norm = sqrtf(part[0]);
        if (!isfinite(norm)) {
            d->gscale = 0.f;               // a non-finite gradient is dropped
            return;
        }
        float scale = 1.f, kept = norm;
        if (d->gnorm_mean > 0.f && norm > clip * d->gnorm_mean) {
            kept = clip * d->gnorm_mean;
            scale = kept / norm;
        }
        d->gnorm_mean = d->gnorm_mean > 0.f ? 0.99f * d->gnorm_mean + 0.01f * kept : norm;
        d->gscale = scale;
    }
}

// Adam (Kingma & Ba 2015) on the FP32 master weights, on the gradient times
// gscale; also folds the step's loss into the epoch total
__global__ void adam_kernel(MlpDev* d, float lr, float b1, float b2, float eps, int t)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) d->loss_epoch += d->loss_sum;
    const float c1 = 1.f - powf(b1, float(t)), c2 = 1.f - powf(b2, float(t));
    const float gs = d->gscale;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < MC_MLP_NWEIGHT;
         k += blockDim.x * gridDim.x) {
        const float gr = d->grad[k] * gs;
        const float m = b1 * d->adam_m[k] + (1.f - b1) * gr;
        const float v = b2 * d->adam_v[k] + (1.f - b2) * gr * gr;
        d->adam_m[k] = m;
        d->adam_v[k] = v;
        d->params[k] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    }
}

// mean / standard deviation of the finite feature rows (FP64 sums): each
// block writes its 21 sums (feature sums, sums of squares, count), reduced
// within the block in a fixed order; set_norm_kernel adds the blocks' sums
// in block order
constexpr int MOMENT_THREADS = 256;
__global__ void __launch_bounds__(MOMENT_THREADS) moments_kernel(long long n, const float* feat,
                                                                 double* sums)
{
    __shared__ double red[MOMENT_THREADS];
    double s[10], q[10], cnt = 0.0;
#pragma unroll
    for (int f = 0; f < 10; f++) s[f] = q[f] = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        bool fin = true;
        float x[10];
#pragma unroll
        for (int f = 0; f < 10; f++) {
            x[f] = feat[i * 10 + f];
            fin = fin && isfinite(x[f]);
        }
        if (!fin) continue;
        cnt += 1.0;
#pragma unroll
        for (int f = 0; f < 10; f++) {
            s[f] += x[f];
            q[f] += double(x[f]) * x[f];
        }
    }
    for (int v = 0; v < 21; v++) {
        red[threadIdx.x] = v < 10 ? s[v] : (v < 20 ? q[v - 10] : cnt);
        __syncthreads();
        for (int w = MOMENT_THREADS / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) sums[(size_t)blockIdx.x * 21 + v] = red[0];
        __syncthreads();
    }
}

__global__ void set_norm_kernel(MlpDev* d, const double* sums, int nblocks)
{
    const int f = threadIdx.x;
    if (f >= 10) return;
    double sf = 0.0, qf = 0.0, c = 0.0;
    for (int b = 0; b < nblocks; b++) {
        sf += sums[(size_t)b * 21 + f];
        qf += sums[(size_t)b * 21 + 10 + f];
        c += sums[(size_t)b * 21 + 20];
    }
    const double cnt = c > 0.0 ? c : 1.0;
    const double mu = sf / cnt;
    const double var = qf / cnt - mu * mu;
    d->params[P_MU + f] = float(mu);
    d->params[P_SIG + f] = float(var > 1e-12 ? sqrt(var) : 1.0);
}

static cudaError_t train_launch(MlpDev* dev, const TrainArgs& a, cudaStream_t s)
{
    int devi = 0, sms = 152;
    cudaGetDevice(&devi);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, devi);
    const long long nchunk = (a.rows + 15) / 16;
    long long blocks = (nchunk + TW - 1) / TW;
    if (blocks > sms) blocks = sms;
    if (blocks > TRAIN_MAX_CTAS) blocks = TRAIN_MAX_CTAS;
    if (blocks < 1) blocks = 1;
    cudaError_t e = cudaFuncSetAttribute(mlp_train_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, TRAIN_SMEM);
    if (e != cudaSuccess) return e;
    mlp_train_kernel<<<(unsigned)blocks, TW * 32, TRAIN_SMEM, s>>>(a);
    if (a.backward)
        reduce_grad_kernel<<<(MC_MLP_NWEIGHT + 255) / 256, 256, 0, s>>>(dev, (int)blocks);
    return cudaGetLastError();
}

}  // namespace mc

using namespace mc;

extern "C" {

mc_status mc_mlp_forward(const mc_mlp* net, int64_t n, const float* features, float* out,
                         void* stream)
{
    if (!net || !features || !out) return set_error(MC_EINVAL, "NULL argument");
    if (n < 0) return set_error(MC_EINVAL, "n < 0");
    if (n == 0) return MC_OK;
    TrainArgs a{net->dev, n, n, 0, 1, 0, features, nullptr, 1.f / float(n), 0, out};
    cudaError_t e = train_launch(net->dev, a, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MC_OK : cuda_error(e, "network forward");
}

mc_status mc_mlp_grad(mc_mlp* net, int64_t n, const float* features, const float* target,
                      float* grads, float* loss, void* stream)
{
    if (!net || !features || !target || !grads || !loss) return set_error(MC_EINVAL, "NULL argument");
    if (n <= 0) return set_error(MC_EINVAL, "n must be > 0");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    zero_grad_kernel<<<(MC_MLP_NWEIGHT + 255) / 256, 256, 0, s>>>(net->dev);
    TrainArgs a{net->dev, n, n, 0, 1, 0, features, target, 1.f / float(n), 1, nullptr};
    cudaError_t e = train_launch(net->dev, a, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(grads, net->dev->grad, sizeof(float) * MC_MLP_NWEIGHT,
                            cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_error(e, "network gradient");
    // loss = sum of squares / n, as float, on the device
    double h = 0.0;
    e = cudaMemcpyAsync(&h, &net->dev->loss_sum, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    float lf = float(h / double(n));
    if (e == cudaSuccess) e = cudaMemcpyAsync(loss, &lf, sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? MC_OK : cuda_error(e, "network gradient");
}

mc_status mc_mlp_train(mc_mlp* net, int64_t n, const float* features, const float* target,
                       const mc_train_cfg* cfg, float* loss_per_epoch, void* stream)
{
    if (!net || !features || !target || !cfg) return set_error(MC_EINVAL, "NULL argument");
    if (n <= 0 || cfg->batch <= 0 || cfg->epochs < 0)
        return set_error(MC_EINVAL, "need n > 0, batch > 0, epochs >= 0");
    if (!(cfg->lr > 0.f) || !(cfg->beta1 >= 0.f && cfg->beta1 < 1.f) ||
        !(cfg->beta2 >= 0.f && cfg->beta2 < 1.f) || !(cfg->eps > 0.f))
        return set_error(MC_EINVAL, "invalid Adam parameters");
    if (!(cfg->clip == 0.f || cfg->clip >= 1.f) || !(cfg->lr_final > 0.f && cfg->lr_final <= cfg->lr))
        return set_error(MC_EINVAL, "need clip = 0 or >= 1 and 0 < lr_final <= lr");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (cfg->fit_norm) {
        double* sums = nullptr;
        long long blocks = (n + MOMENT_THREADS - 1) / MOMENT_THREADS;
        if (blocks > 1024) blocks = 1024;
        e = cudaMallocAsync(&sums, 21 * sizeof(double) * (size_t)blocks, s);
        if (e == cudaSuccess) {
            moments_kernel<<<(unsigned)blocks, MOMENT_THREADS, 0, s>>>(n, features, sums);
            set_norm_kernel<<<1, 32, 0, s>>>(net->dev, sums, (int)blocks);
            e = cudaGetLastError();
            cudaFreeAsync(sums, s);
        }
        if (e != cudaSuccess) return cuda_error(e, "feature standardisation");
    }
    // the Adam step counter lives on the host side of the network's state
    int t = 0;
    e = cudaMemcpyAsync(&t, &net->dev->adam_t, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "reading optimiser state");
    const long long batch = cfg->batch < n ? cfg->batch : n;
    const long long steps = (n + batch - 1) / batch;
    const long long total = steps * cfg->epochs;
    long long done = 0;
    const float one = 1.f;
    e = cudaMemcpyAsync(&net->dev->gscale, &one, sizeof(float), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_error(e, "training set-up");
    uint64_t rs = cfg->seed * 0x9E3779B97F4A7C15ull + 1;
    for (int ep = 0; ep < cfg->epochs; ep++) {
        // row order of this epoch: k -> (a k + b) mod n with gcd(a, n) = 1
        rs = rs * 6364136223846793005ull + 1442695040888963407ull;
        long long pa = (long long)((rs >> 17) % (uint64_t)n);
        if (pa == 0) pa = 1;
        auto gcd = [](long long x, long long y) {
            while (y) {
                long long r = x % y;
                x = y;
                y = r;
            }
            return x;
        };
        while (gcd(pa, n) != 1) pa = pa % n + 1;
        rs = rs * 6364136223846793005ull + 1442695040888963407ull;
        const long long pb = (long long)((rs >> 17) % (uint64_t)n);
        e = cudaMemsetAsync(&net->dev->loss_epoch, 0, sizeof(double), s);
        if (e != cudaSuccess) return cuda_error(e, "training set-up");
        for (long long st = 0; st < steps; st++) {
            const long long first = st * batch;
            const long long rows = (first + batch <= n) ? batch : n - first;
            zero_grad_kernel<<<(MC_MLP_NWEIGHT + 255) / 256, 256, 0, s>>>(net->dev);
            TrainArgs a{net->dev, n, rows, first, pa, pb, features, target,
                        1.f / float(rows), 1, nullptr};
            e = train_launch(net->dev, a, s);
            if (e != cudaSuccess) return cuda_error(e, "training step");
            t++;
            if (cfg->clip > 0.f) clip_kernel<<<1, 256, 0, s>>>(net->dev, cfg->clip);
            // cosine decay from lr to lr_final over the steps of this call
            const double frac = total > 1 ? double(done) / double(total - 1) : 1.0;
            const float lr = float(cfg->lr_final + 0.5 * (cfg->lr - cfg->lr_final) *
                                                       (1.0 + cos(3.141592653589793 * frac)));
            done++;
            adam_kernel<<<(MC_MLP_NWEIGHT + 255) / 256, 256, 0, s>>>(net->dev, lr, cfg->beta1,
                                                                     cfg->beta2, cfg->eps, t);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = mlp_pack(net->dev, s);
            if (e != cudaSuccess) return cuda_error(e, "optimiser step");
        }
        if (loss_per_epoch) {
            double h = 0.0;
            e = cudaMemcpyAsync(&h, &net->dev->loss_epoch, sizeof(double), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_error(e, "reading loss");
            loss_per_epoch[ep] = float(h / double(n));
        }
    }
    e = cudaMemcpyAsync(&net->dev->adam_t, &t, sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? MC_OK : cuda_error(e, "training");
}

}  // extern "C"
