// mc_exact.cu -- exact Euler Riemann solver with plain or learned pressure
// seeds (mc_riemann_exact), and the seed network's device storage.
//
// Toro, ch. 4: p* is the root of f(p) = f_L(p) + f_R(p) + u_R - u_L with
//   f_K(p) = (p - p_K) sqrt(A_K / (p + B_K)),      p > p_K (shock),
//            A_K = 2 / ((gamma+1) rho_K), B_K = (gamma-1)/(gamma+1) p_K,
//   f_K(p) = 2 c_K/(gamma-1) ((p/p_K)^z - 1),      p <= p_K (rarefaction),
//            z = (gamma-1)/(2 gamma),
// and u* = (u_L + u_R)/2 + (f_R(p*) - f_L(p*))/2.  Newton runs in FP64 with
// at most one power per update (p^(z-1), shared by the two sides, and formed
// without FP64 pow when 1/z is an integer, see Powers); seeds are Toro's PV, TR and TS guesses (ch. 9) or the network's proposal
// p_TR exp(net(x)).  One thread per interface; a warp evaluates the network
// for its 32 interfaces together on the tensor cores.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <new>

#include "mc_internal.h"
#include "mc_seednet.cuh"

namespace mc {

constexpr double PFLOOR = 1e-12;

// The powers of the pressure functions, p^-z, p^(z-1) and x^(1/z) with
// z = (gamma-1)/(2 gamma).  When 1/z = 2 gamma/(gamma-1) is an integer n
// (gamma = 1.4: 7; 5/3: 5) they need no FP64 pow: x^(1/z) = x^n by
// repeated squaring, and v = p^(-1/n) by Newton's method on p v^n = 1,
// v <- v + v (1 - p v^n) / n, from an FP32 start (the relative error e
// becomes about (n+1)/2 e^2 per step, so two steps from FP32 reach FP64
// rounding), then p^(z-1) = v^(n-1).  Otherwise, and for p outside
// [1e-30, 1e30], FP64 pow.
struct Powers {
    double z;
    int n;         // 1/z when an integer in [2, 32], else 0
    double invn;   // 1/n
};

__host__ inline Powers make_powers(double gamma)
{
    Powers w;
    w.z = 0.5 * (gamma - 1.0) / gamma;
    const double rz = 2.0 * gamma / (gamma - 1.0);
    const long k = lround(rz);
    w.n = (k >= 2 && k <= 32 && fabs(rz - double(k)) <= 1e-9 * rz) ? int(k) : 0;
    w.invn = w.n ? 1.0 / w.n : 0.0;
    return w;
}

__device__ __forceinline__ double ipow(double v, int k)
{
    double r = 1.0;
    while (k) {
        if (k & 1) r *= v;
        v *= v;
        k >>= 1;
    }
    return r;
}

// p^(-1/n), p > 0
__device__ __forceinline__ double inv_root(const Powers& w, double p)
{
    if (!(p > 1e-30 && p < 1e30)) return pow(p, -w.invn);
    double v = double(powf(float(p), -float(w.invn)));
#pragma unroll
    for (int s = 0; s < 2; s++) v = fma(v * w.invn, fma(-p, ipow(v, w.n), 1.0), v);
    return v;
}

__device__ __forceinline__ double pow_mz(const Powers& w, double p)
{
    return w.n ? inv_root(w, p) : pow(p, -w.z);
}

__device__ __forceinline__ double pow_zm1(const Powers& w, double p)
{
    return w.n ? ipow(inv_root(w, p), w.n - 1) : pow(p, w.z - 1.0);
}

__device__ __forceinline__ double pow_rz(const Powers& w, double x)
{
    if (!w.n) return pow(x, 1.0 / w.z);
    return x > 0.0 ? ipow(x, w.n) : __longlong_as_double(0x7ff8000000000000LL);
}

struct ExactArgs {
    long long n;
    Powers pw;
    double gamma, tol;
    int max_iter, seed_mode;
    const float *rl, *ul, *pl, *rr, *ur, *pr;
    float *ps, *us;
    uint8_t *iters, *flags;
    const MlpDev* net;
    int64_t* stats;
};

struct Side {
    // iA = 1/A_K, ipz = p_K^-z, ikr = p_K^(1-z) / (rho_K c_K)
    double rho, u, p, c, B, iA, kr, ipz, ikr;
};

// One division, one reciprocal square root and one power per side: c and
// 1/c come from the same rsqrt, 1/A_K needs none.
__device__ __forceinline__ Side make_side(double gamma, const Powers& pw, double rho, double u,
                                          double p)
{
    Side s;
    s.rho = rho;
    s.u = u;
    s.p = p;
    const double irho = 1.0 / rho;
    const double c2 = gamma * p * irho;
    const double rc = rsqrt(c2);
    s.c = c2 * rc;
    s.B = (gamma - 1.0) / (gamma + 1.0) * p;
    s.iA = 0.5 * (gamma + 1.0) * rho;
    s.kr = 2.0 * s.c / (gamma - 1.0);
    s.ipz = pow_mz(pw, p);
    s.ikr = irho * rc * p * s.ipz;
    return s;
}

// f_K and f_K' at p; w = p^(z-1) is shared by both sides (only read on the
// rarefaction branch).  Shock: sqrt(A/(B+p)) = rsqrt((B+p)/A) and
// 1/(B+p) = q^2/A.  Rarefaction: (p/p_K)^z = w p p_K^-z and
// f_K' = (p/p_K)^(z-1) / (rho_K c_K) = w p_K^(1-z) / (rho_K c_K).
__device__ __forceinline__ void branch(const Side& s, double p, double w, double& f, double& fd)
{
    if (p > s.p) {
        const double q = rsqrt((s.B + p) * s.iA);
        const double dp = p - s.p;
        f = dp * q;
        fd = q * (1.0 - 0.5 * dp * q * q * s.iA);
    } else {
        f = s.kr * (w * p * s.ipz - 1.0);
        fd = s.ikr * w;
    }
}

// The last Newton evaluation: f_K, f_K' at the iterate p it was taken at.
struct NewtonEval {
    double p, fl, fdl, fr, fdr;
};

// Newton from p0; returns true on convergence, counts updates in it.  The
// power p^(z-1) is formed once per update, and only when a side of some lane
// of the warp is on its rarefaction branch.
__device__ __forceinline__ bool newton(const Side& L, const Side& R, const Powers& pw, double p0,
                                       double tol, int max_iter, double& ps, int& it,
                                       NewtonEval& ev)
{
    double p = p0;
    for (int k = 0; k < max_iter; k++) {
        const double w = (p <= L.p || p <= R.p) ? pow_zm1(pw, p) : 0.0;
        double fl, fdl, fr, fdr;
        branch(L, p, w, fl, fdl);
        branch(R, p, w, fr, fdr);
        ev = NewtonEval{p, fl, fdl, fr, fdr};
        double pn = p - (fl + fr + (R.u - L.u)) / (fdl + fdr);
        if (pn < PFLOOR) pn = PFLOOR;
        it++;
        if (!isfinite(pn)) {
            ps = p;
            return false;
        }
        if (fabs(pn - p) < tol * pn) {   // pn > 0: |dp| / p_{k+1} < tol
            ps = pn;
            return true;
        }
        p = pn;
    }
    ps = p;
    return false;
}

// u* = (u_L + u_R)/2 + (f_R(p*) - f_L(p*))/2 (Toro, ch. 4), with f_K(p*)
// carried from the last Newton evaluation at p to p* to first order: on
// convergence |p* - p| < tol p*, so the omitted term is O(tol^2) of the
// pressure scale.
__device__ __forceinline__ double star_velocity(const Side& L, const Side& R, double ps,
                                                const NewtonEval& ev)
{
    const double d = ps - ev.p;
    return 0.5 * (L.u + R.u) + 0.5 * ((ev.fr - ev.fl) + (ev.fdr - ev.fdl) * d);
}

struct Seeds {
    double pv_raw, pv, tr, ts, adaptive, pvtr;
};

__device__ __forceinline__ Seeds seeds(double gamma, const Powers& pw, const Side& L, const Side& R)
{
    Seeds s;
    const double du = R.u - L.u;
    s.pv_raw = 0.5 * (L.p + R.p) - 0.125 * du * (L.rho + R.rho) * (L.c + R.c);
    s.pv = s.pv_raw < PFLOOR ? PFLOOR : s.pv_raw;
    s.tr = pow_rz(pw, (L.c + R.c - 0.5 * (gamma - 1.0) * du) / (L.c * L.ipz + R.c * R.ipz));
    const double gl = rsqrt((L.B + s.pv) * L.iA), gr = rsqrt((R.B + s.pv) * R.iA);
    s.ts = (gl * L.p + gr * R.p - du) / (gl + gr);
    if (s.ts < PFLOOR) s.ts = PFLOOR;
    const double pmin = fmin(L.p, R.p), pmax = fmax(L.p, R.p);
    const bool pv_ok = pmax / pmin < 2.0 && s.pv >= pmin && s.pv <= pmax;
    s.adaptive = pv_ok ? s.pv : (s.pv < pmin ? s.tr : s.ts);
    s.pvtr = pv_ok ? s.pv : s.tr;
    return s;
}

// The network's ten raw inputs of one interface (FP32), from the FP64 states
// and guesses: ln rho_L, ln rho_R, ln p_L, ln p_R, ln c_L, ln c_R, du,
// du/(c_L + c_R), ln p_TR, ln max(p_PV, 1e-6).
__device__ __forceinline__ void raw_features(const Side& L, const Side& R, const Seeds& sd,
                                             float (&x)[10])
{
    const float du = float(R.u - L.u);
    x[0] = logf(float(L.rho));
    x[1] = logf(float(R.rho));
    x[2] = logf(float(L.p));
    x[3] = logf(float(R.p));
    x[4] = logf(float(L.c));
    x[5] = logf(float(R.c));
    x[6] = du;
    x[7] = du / float(L.c + R.c);
    x[8] = logf(float(sd.tr));
    x[9] = logf(float(fmax(sd.pv_raw, 1e-6)));
}

// ---- The FP32 stage (MC_NEWTON_MIXED).  GB300 runs FP64 at 1/73 of its
// FP32 rate, so Newton first iterates in FP32 from the seed until
// |dp|/p < TOL32, and FP64 updates (newton above, same stopping test
// |p_{k+1} - p_k| / p_{k+1} < tol) finish from there: two of them in the
// usual case, since the FP32 iterate is within about 1e-6 of p* and one FP64
// update squares that relative error.  The FP32 sides, guesses and powers
// use the hardware base-2 logarithm and exponential (relative error a few
// 1e-7), ample for a stage whose result is only a starting point.
constexpr float TOL32 = 1e-5f;
constexpr int MAX32 = 12;

__device__ __forceinline__ float pow32(float x, float y)
{
    float l, r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(x));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y * l));
    return r;
}

struct Side32 {
    float rho, u, p, c, B, iA, kr, ipz, ikr;
};

__device__ __forceinline__ Side32 make_side32(float gamma, float z, float rho, float u, float p)
{
    Side32 s;
    s.rho = rho;
    s.u = u;
    s.p = p;
    const float irho = 1.0f / rho;
    const float c2 = gamma * p * irho;
    const float rc = rsqrtf(c2);
    s.c = c2 * rc;
    s.B = (gamma - 1.0f) / (gamma + 1.0f) * p;
    s.iA = 0.5f * (gamma + 1.0f) * rho;
    s.kr = 2.0f * s.c / (gamma - 1.0f);
    s.ipz = pow32(p, -z);
    s.ikr = irho * rc * p * s.ipz;
    return s;
}

__device__ __forceinline__ void branch32(const Side32& s, float p, float w, float& f, float& fd)
{
    if (p > s.p) {
        const float q = rsqrtf((s.B + p) * s.iA);
        const float dp = p - s.p;
        f = dp * q;
        fd = q * (1.0f - 0.5f * dp * q * q * s.iA);
    } else {
        f = s.kr * (w * p * s.ipz - 1.0f);
        fd = s.ikr * w;
    }
}

struct Seeds32 {
    float pv_raw, pv, tr, ts, adaptive, pvtr;
};

__device__ __forceinline__ Seeds32 seeds32(float gamma, float z, const Side32& L, const Side32& R)
{
    Seeds32 s;
    const float fl = float(PFLOOR);
    const float du = R.u - L.u;
    s.pv_raw = 0.5f * (L.p + R.p) - 0.125f * du * (L.rho + R.rho) * (L.c + R.c);
    s.pv = s.pv_raw < fl ? fl : s.pv_raw;
    const float x = (L.c + R.c - 0.5f * (gamma - 1.0f) * du) / (L.c * L.ipz + R.c * R.ipz);
    s.tr = x > 0.0f ? pow32(x, 1.0f / z) : __int_as_float(0x7fc00000);
    const float gl = rsqrtf((L.B + s.pv) * L.iA), gr = rsqrtf((R.B + s.pv) * R.iA);
    s.ts = (gl * L.p + gr * R.p - du) / (gl + gr);
    if (s.ts < fl) s.ts = fl;
    const float pmin = fminf(L.p, R.p), pmax = fmaxf(L.p, R.p);
    const bool pv_ok = pmax / pmin < 2.0f && s.pv >= pmin && s.pv <= pmax;
    s.adaptive = pv_ok ? s.pv : (s.pv < pmin ? s.tr : s.ts);
    s.pvtr = pv_ok ? s.pv : s.tr;
    return s;
}

__device__ __forceinline__ void raw_features32(const Side32& L, const Side32& R, const Seeds32& sd,
                                               float (&x)[10])
{
    const float du = R.u - L.u;
    x[0] = logf(L.rho);
    x[1] = logf(R.rho);
    x[2] = logf(L.p);
    x[3] = logf(R.p);
    x[4] = logf(L.c);
    x[5] = logf(R.c);
    x[6] = du;
    x[7] = du / (L.c + R.c);
    x[8] = logf(sd.tr);
    x[9] = logf(fmaxf(sd.pv_raw, 1e-6f));
}

// FP32 Newton from p0 until |dp|/p < TOL32 (true) or MAX32 updates (false,
// ps the last finite iterate); updates counted in it.
__device__ __forceinline__ bool newton32(const Side32& L, const Side32& R, float z, float p0,
                                         float& ps, int& it)
{
    float p = p0;
    const float fl = float(PFLOOR);
    for (int k = 0; k < MAX32; k++) {
        const float w = (p <= L.p || p <= R.p) ? pow32(p, z - 1.0f) : 0.0f;
        float f1, d1, f2, d2;
        branch32(L, p, w, f1, d1);
        branch32(R, p, w, f2, d2);
        float pn = p - (f1 + f2 + (R.u - L.u)) / (d1 + d2);
        if (pn < fl) pn = fl;
        it++;
        if (!isfinite(pn)) {
            ps = p;
            return false;
        }
        if (fabsf(pn - p) < TOL32 * pn) {
            ps = pn;
            return true;
        }
        p = pn;
    }
    ps = p;
    return false;
}

// Four CTAs of 128 threads per SM (at most 128 registers a thread): the
// kernel is bound by the FP64 pipe, and 16 resident warps keep it busier
// than the 12 that the uncapped register counts (142-168) allow; measured
// 6-11% more solves/s for the seeded and mixed forms, the same for the plain
// one, which fits in 128 registers anyway.
template <bool MLP, bool MIXED>
__global__ void __launch_bounds__(128, 4) exact_kernel(const ExactArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    MlpShared* net = reinterpret_cast<MlpShared*>(smem);
    __nv_bfloat16* xs = nullptr;
    float* outs = nullptr;
    if (MLP) {
        mlp_load_shared(a.net, net);
        xs = reinterpret_cast<__nv_bfloat16*>(smem + sizeof(MlpShared)) + warp * 32 * XP;
        outs = reinterpret_cast<float*>(smem + sizeof(MlpShared) + 4 * 32 * XP * 2) + warp * 32;
        __syncthreads();
    }
    const double gamma = a.gamma;
    const Powers pw = a.pw;
    long long c_n = 0, c_vac = 0, c_fb = 0, c_nc = 0, c_it = 0, c_max = 0, c_it32 = 0, c_it64 = 0;
    const float g32 = float(gamma), z32 = float(pw.z);
    const long long nchunks = (a.n + 31) / 32;
    for (long long ch = (long long)blockIdx.x * 4 + warp; ch < nchunks;
         ch += (long long)gridDim.x * 4) {
        const long long i = ch * 32 + lane;
        const bool valid = i < a.n;
        Side L, R;
        if (valid) {
            L = make_side(gamma, pw, a.rl[i], a.ul[i], a.pl[i]);
            R = make_side(gamma, pw, a.rr[i], a.ur[i], a.pr[i]);
        } else {
            L = make_side(gamma, pw, 1.0, 0.0, 1.0);
            R = L;
        }
        const bool vacuum = 2.0 / (gamma - 1.0) * (L.c + R.c) <= R.u - L.u;
        int flag = 0, it = 0, it32 = 0;
        double ps = 0.0, p0 = 0.0;
        NewtonEval ev{};
        bool done = false;
        if constexpr (MIXED) {
            // FP32 stage from the seed (or the network's proposal), then FP64
            const Side32 L32 = valid ? make_side32(g32, z32, a.rl[i], a.ul[i], a.pl[i])
                                     : make_side32(g32, z32, 1.0f, 0.0f, 1.0f);
            const Side32 R32 = valid ? make_side32(g32, z32, a.rr[i], a.ur[i], a.pr[i]) : L32;
            const Seeds32 sd = seeds32(g32, z32, L32, R32);
            float p32;
            switch (a.seed_mode & 15) {
            case MC_SEED_PV: p32 = sd.pv; break;
            case MC_SEED_TR: p32 = sd.tr; break;
            case MC_SEED_TS: p32 = sd.ts; break;
            case MC_SEED_PVTR: p32 = sd.pvtr; break;
            default: p32 = sd.adaptive; break;
            }
            float ps32 = 0.0f;
            bool have32 = false;
            if (MLP) {
                float x[10];
                if (!vacuum && valid) {
                    raw_features32(L32, R32, sd, x);
#pragma unroll
                    for (int k = 0; k < 10; k++) x[k] = (x[k] - net->mu[k]) / net->sig[k];
                } else {
#pragma unroll
                    for (int k = 0; k < 10; k++) x[k] = 0.0f;
                }
                const float o = mlp_infer_warp(*net, x, xs, outs);
                if (!vacuum && valid) {
                    const float prop = sd.tr * expf(o);
                    const float pmin = fminf(L32.p, R32.p), pmax = fmaxf(L32.p, R32.p);
                    if (isfinite(prop) && prop >= 1e-6f * pmin && prop <= 1e6f * pmax &&
                        newton32(L32, R32, z32, prop, ps32, it32)) {
                        have32 = true;
                    } else {
                        flag |= MC_RS_FALLBACK;
                        p32 = sd.adaptive;
                    }
                }
            }
            if (valid && !vacuum) {
                if (!have32) {
                    float q = 0.0f;
                    // a stalled FP32 stage still leaves a close start
                    have32 = newton32(L32, R32, z32, p32, q, it32) || (isfinite(q) && q > 0.0f);
                    ps32 = q;
                }
                // FP64 from the FP32 iterate, else from the FP64 adaptive guess
                const double start = have32 ? double(ps32) : seeds(gamma, pw, L, R).adaptive;
                int it64 = 0;
                if (!newton(L, R, pw, start, a.tol, a.max_iter, ps, it64, ev)) flag |= MC_RS_NOCONV;
                done = true;
                it = it32 + it64;
                c_it32 += it32;
                c_it64 += it64;
            }
        } else {
            Seeds sd = seeds(gamma, pw, L, R);
            switch (a.seed_mode) {
            case MC_SEED_PV: p0 = sd.pv; break;
            case MC_SEED_TR: p0 = sd.tr; break;
            case MC_SEED_TS: p0 = sd.ts; break;
            case MC_SEED_PVTR: p0 = sd.pvtr; break;
            default: p0 = sd.adaptive; break;
            }
            if (MLP) {
                float x[10];
                if (!vacuum && valid) {
                    raw_features(L, R, sd, x);
#pragma unroll
                    for (int k = 0; k < 10; k++) x[k] = (x[k] - net->mu[k]) / net->sig[k];
                } else {
#pragma unroll
                    for (int k = 0; k < 10; k++) x[k] = 0.0f;
                }
                const float o = mlp_infer_warp(*net, x, xs, outs);
                if (!vacuum && valid) {
                    // a seed: FP32 accuracy of the factor is ample, and an FP64 exp
                    // would cost as much as a Newton update
                    const double prop = sd.tr * double(expf(o));
                    const double pmin = fmin(L.p, R.p), pmax = fmax(L.p, R.p);
                    if (isfinite(prop) && prop >= 1e-6 * pmin && prop <= 1e6 * pmax &&
                        newton(L, R, pw, prop, a.tol, a.max_iter, ps, it, ev)) {
                        done = true;
                    } else {
                        flag |= MC_RS_FALLBACK;
                        p0 = sd.adaptive;
                    }
                }
            }
        }
        if (valid) {
            if (vacuum) {
                flag = MC_RS_VACUUM;
                it = 0;
                ps = 0.0;
            } else if (!done) {
                if (!newton(L, R, pw, p0, a.tol, a.max_iter, ps, it, ev)) flag |= MC_RS_NOCONV;
            }
            double us = __longlong_as_double(0x7ff8000000000000LL);   // NaN for vacuum
            if (!vacuum) us = star_velocity(L, R, ps, ev);
            a.ps[i] = float(ps);
            a.us[i] = float(us);
            if (a.iters) a.iters[i] = uint8_t(it > 255 ? 255 : it);
            if (a.flags) a.flags[i] = uint8_t(flag);
            c_n++;
            c_vac += vacuum;
            c_fb += (flag & MC_RS_FALLBACK) != 0;
            c_nc += (flag & MC_RS_NOCONV) != 0;
            c_it += it;
            c_max = c_max > it ? c_max : it;
        }
    }
    if (a.stats) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            c_n += __shfl_xor_sync(0xffffffffu, c_n, o);
            c_vac += __shfl_xor_sync(0xffffffffu, c_vac, o);
            c_fb += __shfl_xor_sync(0xffffffffu, c_fb, o);
            c_nc += __shfl_xor_sync(0xffffffffu, c_nc, o);
            c_it += __shfl_xor_sync(0xffffffffu, c_it, o);
            c_it32 += __shfl_xor_sync(0xffffffffu, c_it32, o);
            c_it64 += __shfl_xor_sync(0xffffffffu, c_it64, o);
            long long m = __shfl_xor_sync(0xffffffffu, c_max, o);
            c_max = c_max > m ? c_max : m;
        }
        if (lane == 0) {
            atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[0]), (unsigned long long)c_n);
            atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[1]), (unsigned long long)c_vac);
            atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[2]), (unsigned long long)c_fb);
            atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[3]), (unsigned long long)c_nc);
            atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[4]), (unsigned long long)c_it);
            atomicMax(reinterpret_cast<unsigned long long*>(&a.stats[5]), (unsigned long long)c_max);
            if (MIXED) {
                atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[6]), (unsigned long long)c_it32);
                atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[7]), (unsigned long long)c_it64);
            }
        }
    }
}

constexpr int EXACT_SMEM_MLP = (int)sizeof(MlpShared) + 4 * 32 * XP * 2 + 4 * 32 * 4;

__global__ void features_kernel(long long n, double gamma, Powers pw, const float* rl, const float* ul,
                                const float* pl, const float* rr, const float* ur,
                                const float* pr, const float* ps, float* feat, float* target)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const Side L = make_side(gamma, pw, rl[i], ul[i], pl[i]);
        const Side R = make_side(gamma, pw, rr[i], ur[i], pr[i]);
        const bool vacuum = 2.0 / (gamma - 1.0) * (L.c + R.c) <= R.u - L.u;
        float x[10];
        const Seeds sd = seeds(gamma, pw, L, R);
        raw_features(L, R, sd, x);
        const float nan = __int_as_float(0x7fc00000);
#pragma unroll
        for (int k = 0; k < 10; k++) feat[i * 10 + k] = vacuum ? nan : x[k];
        if (target) {
            const float p = ps[i];
            target[i] = (vacuum || !(p > 0.0f)) ? nan : float(log(double(p)) - log(sd.tr));
        }
    }
}

// BF16 copies of the weights in the fragment-friendly layouts
__global__ void mlp_pack_kernel(MlpDev* d)
{
    for (int k = threadIdx.x + blockIdx.x * blockDim.x; k < NH * W2P;
         k += blockDim.x * gridDim.x) {
        const int r = k / W2P, c = k % W2P;
        // W2 [in j][out k] -> w2t[out][in], w2[in][out]
        d->w2t[k] = __float2bfloat16_rn(c < NH ? d->params[P_W2 + c * NH + r] : 0.0f);
        d->w2[k] = __float2bfloat16_rn(c < NH ? d->params[P_W2 + r * NH + c] : 0.0f);
        if (k < NH * W1P) {
            const int r1 = k / W1P, c1 = k % W1P;
            d->w1t[k] = __float2bfloat16_rn(c1 < 16 ? d->params[P_W1 + c1 * NH + r1] : 0.0f);
        }
        if (k < NH) d->w3r[k] = bf16_round(d->params[P_W3 + k]);
    }
}

cudaError_t mlp_pack(MlpDev* d, cudaStream_t s)
{
    mlp_pack_kernel<<<(NH * W2P + 255) / 256, 256, 0, s>>>(d);
    return cudaGetLastError();
}

}  // namespace mc

using namespace mc;

extern "C" {

mc_status mc_mlp_create(mc_mlp** out)
{
    if (!out) return set_error(MC_EINVAL, "output is NULL");
    *out = nullptr;
    mc_mlp* m = new (std::nothrow) mc_mlp();
    if (!m) return set_error(MC_ENOMEM, "network handle allocation failed");
    cudaError_t e = cudaMalloc(&m->dev, sizeof(MlpDev));
    if (e == cudaSuccess) e = cudaMemset(m->dev, 0, sizeof(MlpDev));
    if (e != cudaSuccess) {
        cudaFree(m->dev);
        delete m;
        return cuda_error(e, "network allocation");
    }
    // unit feature scales until parameters are set
    float ones[10] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1};
    e = cudaMemcpy(m->dev->params + P_SIG, ones, sizeof(ones), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(m->dev);
        delete m;
        return cuda_error(e, "network initialisation");
    }
    *out = m;
    return MC_OK;
}

mc_status mc_mlp_destroy(mc_mlp* m)
{
    if (!m) return MC_OK;
    cudaFree(m->dev);
    delete m;
    return MC_OK;
}

mc_status mc_mlp_set_params(mc_mlp* m, const float* host)
{
    if (!m || !host) return set_error(MC_EINVAL, "NULL argument");
    for (int k = 0; k < 10; k++)
        if (!(host[P_SIG + k] > 0.0f)) return set_error(MC_EINVAL, "feature scale %d must be > 0", k);
    cudaError_t e = cudaMemcpy(m->dev->params, host, sizeof(float) * MC_MLP_NPARAM,
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = mlp_pack(m->dev, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return e == cudaSuccess ? MC_OK : cuda_error(e, "setting network parameters");
}

mc_status mc_mlp_get_params(const mc_mlp* m, float* host)
{
    if (!m || !host) return set_error(MC_EINVAL, "NULL argument");
    cudaError_t e = cudaMemcpy(host, m->dev->params, sizeof(float) * MC_MLP_NPARAM,
                               cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? MC_OK : cuda_error(e, "reading network parameters");
}

mc_status mc_mlp_features(int64_t n, double gamma, const float* rho_l, const float* u_l,
                          const float* p_l, const float* rho_r, const float* u_r,
                          const float* p_r, const float* p_star, float* features, float* target,
                          void* stream)
{
    if (n < 0) return set_error(MC_EINVAL, "n < 0");
    if (n == 0) return MC_OK;
    if (!rho_l || !u_l || !p_l || !rho_r || !u_r || !p_r || !features)
        return set_error(MC_EINVAL, "NULL state or output pointer");
    if (target && !p_star) return set_error(MC_EINVAL, "targets need p_star");
    if (!(gamma > 1.0)) return set_error(MC_EINVAL, "gamma must be > 1");
    long long blocks = (n + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    features_kernel<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        n, gamma, make_powers(gamma), rho_l, u_l, p_l, rho_r, u_r, p_r, p_star, features, target);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MC_OK : cuda_error(e, "features launch");
}

mc_status mc_riemann_exact(int64_t n, double gamma, const float* rho_l, const float* u_l,
                           const float* p_l, const float* rho_r, const float* u_r,
                           const float* p_r, float* p_star, float* u_star, uint8_t* iters,
                           uint8_t* flags, int seed_mode, const mc_mlp* net, double tol,
                           int max_iter, int64_t* stats, void* stream)
{
    if (n < 0) return set_error(MC_EINVAL, "n < 0");
    if (n == 0) return MC_OK;
    if (!rho_l || !u_l || !p_l || !rho_r || !u_r || !p_r || !p_star || !u_star)
        return set_error(MC_EINVAL, "NULL state or output pointer");
    if (!(gamma > 1.0)) return set_error(MC_EINVAL, "gamma must be > 1");
    if (!(tol > 0.0) || max_iter < 1 || max_iter > 255)
        return set_error(MC_EINVAL, "need tol > 0 and 1 <= max_iter <= 255");
    const bool mixed = (seed_mode & MC_NEWTON_MIXED) != 0;
    const int base = seed_mode & ~MC_NEWTON_MIXED;
    if (base < MC_SEED_ADAPTIVE || base > MC_SEED_MLP)
        return set_error(MC_EINVAL, "unknown seed mode %d", seed_mode);
    if (base == MC_SEED_MLP && !net) return set_error(MC_EINVAL, "MLP seed needs a network");
    ExactArgs a{n, make_powers(gamma), gamma, tol, max_iter, base, rho_l, u_l, p_l, rho_r, u_r, p_r,
                p_star, u_star, iters, flags, net ? net->dev : nullptr, stats};
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long nchunks = (n + 31) / 32;
    long long blocks = (nchunks + 3) / 4;
    const long long cap = (long long)sms * 16;
    if (blocks > cap) blocks = cap;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (base == MC_SEED_MLP) {
        cudaError_t e = mixed ? cudaFuncSetAttribute(exact_kernel<true, true>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     EXACT_SMEM_MLP)
                              : cudaFuncSetAttribute(exact_kernel<true, false>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     EXACT_SMEM_MLP);
        if (e != cudaSuccess) return cuda_error(e, "exact solver set-up");
        if (mixed) exact_kernel<true, true><<<(unsigned)blocks, 128, EXACT_SMEM_MLP, s>>>(a);
        else exact_kernel<true, false><<<(unsigned)blocks, 128, EXACT_SMEM_MLP, s>>>(a);
    } else if (mixed) {
        exact_kernel<false, true><<<(unsigned)blocks, 128, 0, s>>>(a);
    } else {
        exact_kernel<false, false><<<(unsigned)blocks, 128, 0, s>>>(a);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MC_OK : cuda_error(e, "exact solver launch");
}

}  // extern "C"
