// mc_riemann.cuh -- pointwise Riemann solvers of the GPU path.
//
// The paper (§1.1, §2) keeps the Riemann solver pointwise and unaware of the
// parallelism around it; Table 1 gives its data flow (cell-centre states in,
// edge values out).  Each solver here maps the two states adjacent to one
// edge to waves W^p, speeds s^p and the fluctuations A-dQ, A+dQ, and keeps the
// linearised (Roe) state of the edge so the transverse split can reuse it.
// Mathematics: LeVeque (2002) §3.9 (acoustics), §15.3.3-15.3.5 (Roe solvers
// for shallow water and Euler, Harten-Hyman entropy fix), §21.2 (transverse
// split).  Template parameter DIR is the edge normal: 0 = x, 1 = y; the
// normal momentum is component 1 + DIR and the tangential one 2 - DIR.
#pragma once

#include <cuda_runtime.h>

namespace mc {

template <typename T>
__device__ __forceinline__ T tmin0(T a) { return a < T(0) ? a : T(0); }
template <typename T>
__device__ __forceinline__ T tmax0(T a) { return a > T(0) ? a : T(0); }

// Reciprocal, square root and reciprocal square root.  FP32 uses the
// hardware approximations (rcp/sqrt/rsqrt.approx: at most about 2 ulp, far
// inside the FP32 parity tolerance); FP64 keeps correctly rounded square
// roots and reciprocals, so every kernel that inlines them gets the same
// bits (an FP64 rsqrt is not correctly rounded, and its inlined form
// differed between kernels).
__device__ __forceinline__ float rcp_(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double rcp_(double x) { return __drcp_rn(x); }
__device__ __forceinline__ float rsqrt_(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double rsqrt_(double x) { return __drcp_rn(__dsqrt_rn(x)); }
__device__ __forceinline__ float sqrt_(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
// x^y for x > 0: FP32 as 2^(y log2 x) with the hardware base-2 approximations
// (relative error a few ulp for the moderate exponents used here), FP64 pow
__device__ __forceinline__ float pow_(float x, float y)
{
    float l, r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(x));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y * l));
    return r;
}
__device__ __forceinline__ double pow_(double x, double y) { return pow(x, y); }

// Packed FP32 pairs.  One iteration of the sweep solves an x-edge and a
// y-edge with the same arithmetic; written in the edge-normal frame
// (component 1 the normal momentum or velocity, 2 the tangential one) the two
// solves are identical, so FP32 runs them side by side in the halves of a
// float2 with the packed add/multiply/fma instructions of sm_100 and later:
// one issue slot per pair instead of two.  Each half rounds like the scalar
// instruction (round to nearest even), so a packed result equals the scalar
// result of the same operation sequence.
using f2 = float2;
__device__ __forceinline__ f2 p_set(float a) { return make_float2(a, a); }
__device__ __forceinline__ f2 p_add(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 p_mul(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 p_fma(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
// a - b as b (-1) + a: the product is exact, so one rounding like a - b
__device__ __forceinline__ f2 p_sub(f2 a, f2 b) { return __ffma2_rn(b, p_set(-1.f), a); }
__device__ __forceinline__ f2 p_neg(f2 a) { return p_mul(a, p_set(-1.f)); }
__device__ __forceinline__ f2 p_rcp(f2 a) { return make_float2(rcp_(a.x), rcp_(a.y)); }
__device__ __forceinline__ f2 p_rsqrt(f2 a) { return make_float2(rsqrt_(a.x), rsqrt_(a.y)); }
__device__ __forceinline__ f2 p_sqrt(f2 a) { return make_float2(sqrt_(a.x), sqrt_(a.y)); }
__device__ __forceinline__ f2 p_min0(f2 a) { return make_float2(tmin0(a.x), tmin0(a.y)); }
__device__ __forceinline__ f2 p_max0(f2 a) { return make_float2(tmax0(a.x), tmax0(a.y)); }
__device__ __forceinline__ float half(const f2& a, int h) { return h ? a.y : a.x; }
__device__ __forceinline__ float& half(f2& a, int h) { return h ? a.y : a.x; }

// Edge-normal frame: component m of the frame is component frame_comp(m, DIR)
// of the physical state (the two momenta swap for a y-edge).
__host__ __device__ constexpr int frame_comp(int m, int dir)
{
    return dir == 0 ? m : (m == 1 ? 2 : (m == 2 ? 1 : m));
}

// ---------------------------------------------------------------- acoustics
template <typename T>
struct AcousticsRP {
    using real = T;
    static constexpr int NEQ = 3, NW = 2;
    static constexpr int NAUX = 0, NPLANE = NEQ;   // state planes: the conserved fields
    static constexpr bool POSITIVE = false;   // no positivity constraint on (p, u, v)
    T c, Z, inv2Z;
    bool efix;  // unused: linear system
    struct Lin {};
    // component m of wave p can be non-zero (the tangential velocity never is)
    template <int DIR>
    __host__ __device__ static constexpr bool wave_nz(int, int m) { return m != 2 - DIR; }
    // the sweep keeps the y-edge waves of the row below (not their products)
    static constexpr bool CARRY_DOT = false;
    static constexpr bool PAIRED = false;   // scalar solves only
    static constexpr bool SEEDED = false;   // no external pressure seed

    __device__ __forceinline__ void cell_speeds(const T*, T& sx, T& sy) const { sx = sy = c; }
    // max over the edge's waves of |s| (the speeds are -c, +c)
    __device__ __forceinline__ T max_speed(const Lin&) const { return c; }

    __host__ void setup(const double* param, int /*efix*/)
    {
        double rho = param[0], K = param[1];
        double cc = sqrt(K / rho);
        c = T(cc);
        Z = T(rho * cc);
        inv2Z = T(0.5 / (rho * cc));
        efix = false;
    }

    template <int DIR>
    __device__ __forceinline__ void normal(const T* ql, const T* qr, T (&W)[NW][NEQ], T (&s)[NW],
                                           T* amdq, T* apdq, Lin&, bool&) const
    {
        constexpr int un = 1 + DIR, ut = 2 - DIR;
        T dp = qr[0] - ql[0], du = qr[un] - ql[un];
        T a1 = (Z * du - dp) * inv2Z;
        T a2 = (dp + Z * du) * inv2Z;
        W[0][0] = -Z * a1; W[0][un] = a1; W[0][ut] = T(0);
        W[1][0] = Z * a2;  W[1][un] = a2; W[1][ut] = T(0);
        s[0] = -c;
        s[1] = c;
        amdq[0] = -c * W[0][0]; amdq[un] = -c * a1; amdq[ut] = T(0);
        apdq[0] = c * W[1][0];  apdq[un] = c * a2;  apdq[ut] = T(0);
    }

    // split a fluctuation of a DIR-normal edge in direction 1 - DIR
    template <int DIR>
    __device__ __forceinline__ void transverse(const Lin&, const T* a, T* bm, T* bp) const
    {
        constexpr int vn = 2 - DIR, vt = 1 + DIR;
        T b1 = (Z * a[vn] - a[0]) * inv2Z;
        T b2 = (a[0] + Z * a[vn]) * inv2Z;
        bm[0] = c * Z * b1;  bm[vn] = -c * b1; bm[vt] = T(0);
        bp[0] = c * Z * b2;  bp[vn] = c * b2;  bp[vt] = T(0);
    }
};

// ---------------------------------------------------------------- acoustics, variable coefficients
// Density rho and sound speed c per cell, carried as state planes 3 and 4
// after (p, u, v) and copied unchanged by the step (the paper's
// variable-coefficient acoustics, §3 Table 2).  The normal solve puts the
// left-going wave on the left medium's eigenvector (-Z_l, 1, 0) at speed -c_l
// and the right-going one on the right medium's (Z_r, 1, 0) at +c_r
// (LeVeque 2002, §9.6).  The transverse split of a fluctuation entering a
// cell takes, toward each neighbour across the split direction, the
// component along that neighbour's outgoing eigenvector at the interface
// between the two cells; reflections there are why the parts do not add up.
template <typename T>
struct AcousticsVarRP {
    using real = T;
    static constexpr int NEQ = 3, NW = 2;
    static constexpr int NAUX = 2, NPLANE = NEQ + NAUX;
    static constexpr bool POSITIVE = false;
    template <int DIR>
    __host__ __device__ static constexpr bool wave_nz(int, int m) { return m != 2 - DIR; }
    static constexpr bool CARRY_DOT = false;
    static constexpr bool PAIRED = false;   // scalar solves only
    static constexpr bool SEEDED = false;   // no external pressure seed
    bool efix;  // unused: linear
    struct Lin { T cl, cr; };
    __device__ __forceinline__ T max_speed(const Lin& L) const { return fmax(L.cl, L.cr); }
    __device__ __forceinline__ void cell_speeds(const T* q, T& sx, T& sy) const { sx = sy = q[4]; }
    __host__ void setup(const double*, int) { efix = false; }

    template <int DIR>
    __device__ __forceinline__ void normal(const T* ql, const T* qr, T (&W)[NW][NEQ], T (&s)[NW],
                                           T* amdq, T* apdq, Lin& L, bool&) const
    {
        constexpr int un = 1 + DIR, ut = 2 - DIR;
        const T zl = ql[3] * ql[4], zr = qr[3] * qr[4];
        const T dp = qr[0] - ql[0], du = qr[un] - ql[un];
        const T rz = rcp_(zl + zr);
        const T a1 = (zr * du - dp) * rz, a2 = (zl * du + dp) * rz;
        W[0][0] = -zl * a1; W[0][un] = a1; W[0][ut] = T(0);
        W[1][0] = zr * a2;  W[1][un] = a2; W[1][ut] = T(0);
        s[0] = -ql[4];
        s[1] = qr[4];
        amdq[0] = s[0] * W[0][0]; amdq[un] = s[0] * a1; amdq[ut] = T(0);
        apdq[0] = s[1] * W[1][0]; apdq[un] = s[1] * a2; apdq[ut] = T(0);
        L.cl = ql[4];
        L.cr = qr[4];
    }

    // a enters the cell with material (rho, c) = mid; lo and hi are its
    // neighbours across the split direction (below/above for an x-edge's
    // fluctuation, DIR = 0; left/right for a y-edge's, DIR = 1)
    template <int DIR>
    __device__ __forceinline__ void transverse_cells(const T* lo, const T* mid, const T* hi, const T* a,
                                                     T* bm, T* bp) const
    {
        constexpr int vn = 2 - DIR, vt = 1 + DIR;
        const T zlo = lo[0] * lo[1], z = mid[0] * mid[1], zhi = hi[0] * hi[1];
        const T dn = (z * a[vn] - a[0]) * rcp_(zlo + z);
        const T up = (z * a[vn] + a[0]) * rcp_(z + zhi);
        bm[0] = lo[1] * zlo * dn; bm[vn] = -lo[1] * dn; bm[vt] = T(0);
        bp[0] = hi[1] * zhi * up; bp[vn] = hi[1] * up;  bp[vt] = T(0);
    }
};

// ---------------------------------------------------------------- advection
// q_t + u q_x + v q_y = 0 with constant velocity (u, v) = (param[0],
// param[1]): one wave, the jump, moving at the edge-normal velocity
// (LeVeque 2002, §4.8, §20.1); the transverse velocity carries a fluctuation
// across the other edges (§20.2).
template <typename T>
struct AdvectionRP {
    using real = T;
    static constexpr int NEQ = 1, NW = 1;
    static constexpr int NAUX = 0, NPLANE = NEQ;
    static constexpr bool POSITIVE = false;
    template <int DIR>
    __host__ __device__ static constexpr bool wave_nz(int, int) { return true; }
    static constexpr bool CARRY_DOT = false;
    static constexpr bool PAIRED = false;   // scalar solves only
    static constexpr bool SEEDED = false;   // no external pressure seed
    T u, v;
    bool efix;  // unused: linear
    struct Lin { T s; };
    __device__ __forceinline__ T max_speed(const Lin& L) const { return fabs(L.s); }
    __device__ __forceinline__ void cell_speeds(const T*, T& sx, T& sy) const
    {
        sx = fabs(u);
        sy = fabs(v);
    }
    __host__ void setup(const double* param, int)
    {
        u = T(param[0]);
        v = T(param[1]);
        efix = false;
    }
    template <int DIR>
    __device__ __forceinline__ void normal(const T* ql, const T* qr, T (&W)[NW][NEQ], T (&s)[NW],
                                           T* amdq, T* apdq, Lin& L, bool&) const
    {
        const T sn = DIR == 0 ? u : v;
        W[0][0] = qr[0] - ql[0];
        s[0] = sn;
        amdq[0] = tmin0(sn) * W[0][0];
        apdq[0] = tmax0(sn) * W[0][0];
        L.s = sn;
    }
    template <int DIR>
    __device__ __forceinline__ void transverse(const Lin&, const T* a, T* bm, T* bp) const
    {
        const T st = DIR == 0 ? v : u;
        bm[0] = tmin0(st) * a[0];
        bp[0] = tmax0(st) * a[0];
    }
};

// ---------------------------------------------------------------- FP64 guard
// FP32 runs recompute a few edges in FP64: edges across a near-dry or
// near-vacuum front (the smaller depth or density below tau times the
// larger), Euler edges whose Roe sound speed is a vanishing part of the
// enthalpy (c^2 < tau (gamma - 1) H: cold, high-Mach flow, where c^2 is the
// difference of two nearly equal terms), and the speeds and the split of a
// transonic entropy fix.  An Edge64 carries one such edge's results, in the
// edge-normal frame (component 1 the normal momentum), rounded to FP32.
struct Edge64 {
    float W[3][4];
    float s[3];
    float am[4], ap[4];
    float lin[6];             // the linearised state (solver's Lin fields in order)
    float tm[4], tp[4];       // transverse split of am (B-, B+)
    float um[4], up[4];       // ... and of ap
    bool bad;
};
// the normal solve (and, with trans, both transverse splits) of one edge in
// FP64; a and b are the left and right states in the edge-normal frame
static __device__ __forceinline__ Edge64 swe_edge64(double g, bool efix, const float (&a)[3],
                                                 const float (&b)[3], bool trans);
static __device__ __forceinline__ Edge64 euler_edge64(double gamma, bool efix, const float (&a)[4],
                                                   const float (&b)[4], bool trans);
// default relative threshold of the guard (param[3] = 0)
constexpr float GUARD_TAU_DEFAULT = 1e-3f;

// ---------------------------------------------------------------- shallow water
template <typename T>
struct SweRP {
    using real = T;
    static constexpr int NEQ = 3, NW = 3;
    static constexpr int NAUX = 0, NPLANE = NEQ;
    static constexpr bool POSITIVE = true;    // depth h > 0
    T g;
    bool efix;
    double gd;        // g in FP64 (guarded edges)
    float gtau;       // FP32 guard threshold; negative: guard off
    struct Lin { T u, v, c, r2c; };
    // component m of wave p can be non-zero: the shear wave moves only the
    // tangential momentum
    template <int DIR>
    __host__ __device__ static constexpr bool wave_nz(int p, int m) { return p != 1 || m == 2 - DIR; }
    // the sweep carries the limiter dot products of the y-edge waves with
    // those of the row below (measured 1-3% faster than carrying the waves)
    static constexpr bool CARRY_DOT = true;
    // max over the edge's waves of |s|: speeds u - c, u, u + c with c > 0
    __device__ __forceinline__ T max_speed(const Lin& L) const { return fabs(L.u) + L.c; }

    __device__ __forceinline__ void cell_speeds(const T* q, T& sx, T& sy) const
    {
        const T c = sqrt(g * q[0]);
        sx = fabs(q[1] / q[0]) + c;
        sy = fabs(q[2] / q[0]) + c;
    }

    __host__ void setup(const double* param, int ef)
    {
        g = T(param[0]);
        efix = ef != 0;
        gd = param[0];
        gtau = param[3] == 0.0 ? GUARD_TAU_DEFAULT : float(param[3]);
    }
    __host__ __device__ __forceinline__ bool guard_on() const { return sizeof(T) == 4 && gtau >= 0.f; }
    // an edge across a near-dry front: the smaller depth below gtau times
    // the larger
    __device__ __forceinline__ bool near_dry(float hl, float hr) const
    {
        return (hl < gtau * hr) | (hr < gtau * hl);
    }
    // Harten-Hyman for a wave with states (ha, hua) on its left and (hb,
    // hub) on its right, characteristic speed hu/h + sg sqrt(g h) (sg = -1:
    // the 1-wave, +1: the 3-wave), Roe speed sroe: if the speeds straddle
    // zero, k = beta lam_a with beta = (lam_b - sroe) / (lam_b - lam_a), the
    // left-going part; otherwise k is left as it is.  F64: the speeds and
    // the split in FP64 (the guard's recompute of an FP32 step).
    // Returns true (FP32 form) when a speed lies within gtau times cref (the
    // Roe sound speed) of zero: a near-sonic edge for the FP64 guard.
    template <bool F64 = false>
    __device__ __forceinline__ bool hh_fix(T ha, T hua, T hb, T hub, T sg, T sroe, T cref, T& k) const
    {
        if constexpr (F64) {
            const double la = double(hua) / double(ha) + double(sg) * sqrt(gd * double(ha));
            const double lb = double(hub) / double(hb) + double(sg) * sqrt(gd * double(hb));
            if (la < 0.0 && lb > 0.0) k = T((lb - double(sroe)) / (lb - la) * la);
            return false;
        } else {
            const T la = hua * rcp_(ha) + sg * sqrt_(g * ha);
            const T lb = hub * rcp_(hb) + sg * sqrt_(g * hb);
            if (la < T(0) && lb > T(0)) k = (lb - sroe) * rcp_(lb - la) * la;
            return fabs(la) < T(gtau) * cref || fabs(lb) < T(gtau) * cref;
        }
    }

    // the sweep may pass each state's 1/sqrt(h), formed once per cell
    static constexpr bool RS_CACHE = true;
    __device__ __forceinline__ T rs_of(const T* q) const { return rsqrt_(q[0]); }

    template <int DIR>
    __device__ __forceinline__ void normal(const T* ql, const T* qr, T (&W)[NW][NEQ], T (&s)[NW],
                                           T* amdq, T* apdq, Lin& L, bool& bad) const
    {
        normal_rs<DIR>(ql, qr, rsqrt_(ql[0]), rsqrt_(qr[0]), W, s, amdq, apdq, L, bad);
    }

    // the normal solve given rsl = 1/sqrt(h_l) and rsr = 1/sqrt(h_r)
    template <int DIR>
    __device__ __forceinline__ void normal_rs(const T* ql, const T* qr, T rsl, T rsr, T (&W)[NW][NEQ],
                                              T (&s)[NW], T* amdq, T* apdq, Lin& L, bool& bad) const
    {
        constexpr int un = 1 + DIR, ut = 2 - DIR;
        const T hl = ql[0], hr = qr[0];
        // a non-positive depth is flagged; the arithmetic then yields NaNs,
        // which the caller's status word reports
        bad = bad || !(hl > T(0) && hr > T(0));
        // Roe average: sqrt(h) u = hu / sqrt(h), so one reciprocal square
        // root per state gives both weights
        const T w = rcp_(hl * rsl + hr * rsr);
        const T u = (ql[un] * rsl + qr[un] * rsr) * w;
        const T v = (ql[ut] * rsl + qr[ut] * rsr) * w;
        const T gh = g * T(0.5) * (hl + hr);
        const T rc = rsqrt_(gh);
        const T c = gh * rc;
        const T r2c = T(0.5) * rc;
        const T d0 = hr - hl, dn = qr[un] - ql[un], dt = qr[ut] - ql[ut];
        const T a1 = ((u + c) * d0 - dn) * r2c;
        const T a2 = dt - v * d0;
        const T a3 = (dn - (u - c) * d0) * r2c;
        W[0][0] = a1; W[0][un] = a1 * (u - c); W[0][ut] = a1 * v;
        W[1][0] = T(0); W[1][un] = T(0); W[1][ut] = a2;
        W[2][0] = a3; W[2][un] = a3 * (u + c); W[2][ut] = a3 * v;
        s[0] = u - c;
        s[1] = u;
        s[2] = u + c;
        L.u = u; L.v = v; L.c = c; L.r2c = r2c;

        T k0 = tmin0(s[0]), k2 = tmin0(s[2]);
        if (efix) {
            // Harten-Hyman: a nonlinear wave is transonic when the
            // characteristic speed on its left is negative and on its right
            // positive.  The signs of u -+ sqrt(g h) are decided without a
            // square root or division (u < c  <=>  hu <= 0 or (hu)^2 < g h^3);
            // only a transonic wave pays for the speeds themselves.  A
            // non-positive intermediate depth leaves the wave unfixed.
            // The test of the intermediate state (faster than sound) comes
            // first: it rarely holds, and the outer state's test is then
            // skipped.
            const T hul = ql[un], hum = ql[un] + W[0][un], hm = hl + W[0][0];
            if (hm > T(0) && hum > T(0) && hum * hum > g * hm * hm * hm) {
                if (hul <= T(0) || hul * hul < g * hl * hl * hl) hh_fix(hl, hul, hm, hum, T(-1), s[0], c, k0);
            }
            const T hur = qr[un], hun = qr[un] - W[2][un], hn = hr - W[2][0];
            if (hn > T(0) && hun < T(0) && hun * hun > g * hn * hn * hn) {
                if (hur >= T(0) || hur * hur < g * hr * hr * hr) hh_fix(hn, hun, hr, hur, T(1), s[2], c, k2);
            }
        }
        // A-dQ = sum_p k_p W^p, A+dQ = sum_p (s^p - k_p) W^p (k_p = min(s^p, 0)
        // unless the entropy fix replaced it), over the non-zero components
        const T k1 = tmin0(s[1]);
        const T m2 = k1 * a2, p2 = (s[1] - k1) * a2;
        if (k0 == s[0] && k2 == T(0) && s[2] > T(0)) {
            // subsonic, no fix: wave 1 is all left-going, wave 3 all
            // right-going; the sums below without their zero terms
            const T m1 = k0 * a1, p3 = s[2] * a3;
            amdq[0] = m1;
            amdq[un] = m1 * (u - c);
            amdq[ut] = m1 * v + m2;
            apdq[0] = p3;
            apdq[un] = p3 * (u + c);
            apdq[ut] = p3 * v + p2;
            return;
        }
        const T m1 = k0 * a1, m3 = k2 * a3;
        const T p1 = (s[0] - k0) * a1, p3 = (s[2] - k2) * a3;
        amdq[0] = m1 + m3;
        amdq[un] = m1 * (u - c) + m3 * (u + c);
        amdq[ut] = (m1 + m3) * v + m2;
        apdq[0] = p1 + p3;
        apdq[un] = p1 * (u - c) + p3 * (u + c);
        apdq[ut] = (p1 + p3) * v + p2;
    }

    // ---- FP32 pairs: half .x an x-edge, .y a y-edge, both in the
    // edge-normal frame (component 1 normal, 2 tangential momentum); the
    // same arithmetic as normal<0> / transverse<0>, two edges per instruction
    static constexpr bool PAIRED = sizeof(T) == 4;
    static constexpr bool SEEDED = false;   // no external pressure seed
    // FP32: three resident CTAs of four warps per SM (at most 168 registers)
    static constexpr int MIN_CTAS = sizeof(T) == 4 ? 3 : 1;
    struct LinP { f2 u, v, c, r2c; };
    // the scalar linearised state of half h (x-edge 0, y-edge 1)
    __device__ __forceinline__ Lin lin_half(const LinP& P, int h) const
    {
        return Lin{half(P.u, h), half(P.v, h), half(P.c, h), half(P.r2c, h)};
    }
    __device__ __forceinline__ float max_speed(const LinP& L, int h) const
    {
        return fabs(half(L.u, h)) + half(L.c, h);
    }

    // hh: bit h set when half h met a near-sonic transonic wave (a speed
    // within gtau times the Roe sound speed of zero); F64FIX: the transonic
    // fix's speeds and split in FP64
    template <bool F64FIX = false>
    __device__ __forceinline__ void normal_pair(const f2* ql, const f2* qr, f2 (&W)[NW][NEQ],
                                                f2 (&s)[NW], f2* amdq, f2* apdq, LinP& L,
                                                bool& badx, bool& bady, int& hh) const
    {
        const f2 hl = ql[0], hr = qr[0];
        badx = badx || !(hl.x > 0.f && hr.x > 0.f);
        bady = bady || !(hl.y > 0.f && hr.y > 0.f);
        const f2 rsl = p_rsqrt(hl), rsr = p_rsqrt(hr);
        const f2 w = p_rcp(p_fma(hl, rsl, p_mul(hr, rsr)));
        const f2 u = p_mul(p_fma(ql[1], rsl, p_mul(qr[1], rsr)), w);
        const f2 v = p_mul(p_fma(ql[2], rsl, p_mul(qr[2], rsr)), w);
        const f2 gh = p_mul(p_set(g * 0.5f), p_add(hl, hr));
        const f2 rc = p_rsqrt(gh);
        const f2 c = p_mul(gh, rc);
        const f2 r2c = p_mul(p_set(0.5f), rc);
        const f2 d0 = p_sub(hr, hl), ndn = p_sub(ql[1], qr[1]), dt = p_sub(qr[2], ql[2]);
        const f2 sm = p_sub(u, c), sp = p_add(u, c);
        // a1 = ((u + c) d0 - dn) / 2c, a2 = dt - v d0, a3 = (dn - (u - c) d0) / 2c
        const f2 a1 = p_mul(p_fma(sp, d0, ndn), r2c);
        const f2 a2 = p_fma(p_neg(v), d0, dt);
        const f2 a3 = p_mul(p_fma(sm, d0, ndn), p_neg(r2c));
        W[0][0] = a1; W[0][1] = p_mul(a1, sm); W[0][2] = p_mul(a1, v);
        W[1][0] = p_set(0.f); W[1][1] = p_set(0.f); W[1][2] = a2;
        W[2][0] = a3; W[2][1] = p_mul(a3, sp); W[2][2] = p_mul(a3, v);
        s[0] = sm;
        s[1] = u;
        s[2] = sp;
        L.u = u; L.v = v; L.c = c; L.r2c = r2c;

        f2 k0 = p_min0(sm), k2 = p_min0(sp);
        if (efix) {
            // the transonic tests of normal(), both halves at once.  A wave
            // can be transonic only if its intermediate state moves faster
            // than sound (rightward for the 1-wave, leftward for the 3-wave);
            // those two tests come first, and the tests of the outer states
            // only for a lane where one of them holds
            const f2 gs = p_set(g);
            const f2 hum = p_add(ql[1], W[0][1]), hm = p_add(hl, a1);
            const f2 hun = p_sub(qr[1], W[2][1]), hn = p_sub(hr, a3);
            const f2 hum2 = p_mul(hum, hum), gm3 = p_mul(p_mul(p_mul(gs, hm), hm), hm);
            const f2 hun2 = p_mul(hun, hun), gn3 = p_mul(p_mul(p_mul(gs, hn), hn), hn);
            bool r_pos[2], n_neg[2];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                r_pos[h] = (half(hm, h) > 0.f) & (half(hum, h) > 0.f) & (half(hum2, h) > half(gm3, h));
                n_neg[h] = (half(hn, h) > 0.f) & (half(hun, h) < 0.f) & (half(hun2, h) > half(gn3, h));
            }
            if (r_pos[0] | r_pos[1] | n_neg[0] | n_neg[1]) {
                const f2 hul = ql[1], hur = qr[1];
                const f2 hul2 = p_mul(hul, hul), gl3 = p_mul(p_mul(p_mul(gs, hl), hl), hl);
                const f2 hur2 = p_mul(hur, hur), gr3 = p_mul(p_mul(p_mul(gs, hr), hr), hr);
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const bool l_neg = (half(hul, h) <= 0.f) | (half(hul2, h) < half(gl3, h));
                    const bool rr_pos = (half(hur, h) >= 0.f) | (half(hur2, h) < half(gr3, h));
                    if (l_neg & r_pos[h]) {
                        if (hh_fix<F64FIX>(half(hl, h), half(hul, h), half(hm, h), half(hum, h), -1.f,
                                           half(sm, h), half(c, h), half(k0, h)))
                            hh |= 1 << h;
                    }
                    if (n_neg[h] & rr_pos) {
                        if (hh_fix<F64FIX>(half(hn, h), half(hun, h), half(hr, h), half(hur, h), 1.f,
                                           half(sp, h), half(c, h), half(k2, h)))
                            hh |= 1 << h;
                    }
                }
            }
        }
        const f2 k1 = p_min0(u);
        const f2 m1 = p_mul(k0, a1), m2 = p_mul(k1, a2), m3 = p_mul(k2, a3);
        const f2 q1 = p_mul(p_sub(sm, k0), a1), q2 = p_mul(p_max0(u), a2), q3 = p_mul(p_sub(sp, k2), a3);
        amdq[0] = p_add(m1, m3);
        amdq[1] = p_fma(m1, sm, p_mul(m3, sp));
        amdq[2] = p_fma(amdq[0], v, m2);
        apdq[0] = p_add(q1, q3);
        apdq[1] = p_fma(q1, sm, p_mul(q3, sp));
        apdq[2] = p_fma(apdq[0], v, q2);
    }

    // SUB: the subsonic form below (a caller near its register cap may
    // leave it out)
    template <bool SUB = true>
    __device__ __forceinline__ void transverse_pair(const LinP& L, const f2* a, f2* bm, f2* bp) const
    {
        // transverse<0> in the edge-normal frame: split direction normal
        // component 2, tangential 1
        const f2 u = L.v, v = L.u, c = L.c;
        const f2 l1 = p_sub(u, c), l3 = p_add(u, c);
        // b1 = ((u + c) a0 - a2) / 2c, b2 = a1 - v a0, b3 = (a2 - (u - c) a0) / 2c
        const f2 b1 = p_mul(p_fma(p_neg(l3), a[0], a[2]), p_neg(L.r2c));
        const f2 b2 = p_fma(p_neg(v), a[0], a[1]);
        const f2 b3 = p_mul(p_fma(p_neg(l1), a[0], a[2]), L.r2c);
        const f2 m2 = p_mul(p_min0(u), b2), q2 = p_mul(p_max0(u), b2);
        if (SUB && (l1.x < 0.f) & (l1.y < 0.f) & (l3.x > 0.f) & (l3.y > 0.f)) {
            // both halves subsonic across the split direction (the common
            // case): wave 1 all to B-, wave 3 all to B+; the sums below
            // without their zero terms
            const f2 m1 = p_mul(l1, b1), q3 = p_mul(l3, b3);
            bm[0] = m1;
            bm[2] = p_mul(m1, l1);
            bm[1] = p_fma(m1, v, m2);
            bp[0] = q3;
            bp[2] = p_mul(q3, l3);
            bp[1] = p_fma(q3, v, q2);
            return;
        }
        const f2 m1 = p_mul(p_min0(l1), b1), m3 = p_mul(p_min0(l3), b3);
        const f2 q1 = p_mul(p_max0(l1), b1), q3 = p_mul(p_max0(l3), b3);
        bm[0] = p_add(m1, m3);
        bm[2] = p_fma(m1, l1, p_mul(m3, l3));
        bm[1] = p_fma(bm[0], v, m2);
        bp[0] = p_add(q1, q3);
        bp[2] = p_fma(q1, l1, p_mul(q3, l3));
        bp[1] = p_fma(bp[0], v, q2);
    }

    // The FP64 guard of a pair: bit h set when half h is a near-dry edge.
    __device__ __forceinline__ int guard_mask(const f2* ql, const f2* qr, const LinP&) const
    {
        if (!guard_on()) return 0;
        const f2 tl = p_mul(ql[0], p_set(gtau)), tr = p_mul(qr[0], p_set(gtau));
        return ((ql[0].x < tr.x) | (qr[0].x < tl.x)) | (((ql[0].y < tr.y) | (qr[0].y < tl.y)) << 1);
    }
    // Replaces the results of the guarded halves by their FP64 solve (and,
    // with trans, their FP64 transverse splits).
    __device__ __forceinline__ void guard_redo(const f2* ql, const f2* qr, int gm, bool trans,
                                               f2 (&W)[NW][NEQ], f2 (&s)[NW], f2* am, f2* ap,
                                               LinP& L, f2* Tm, f2* Tp, f2* Um, f2* Up, bool& badx,
                                               bool& bady) const
    {
#pragma unroll
        for (int h = 0; h < 2; h++) {
            if (!((gm >> h) & 1)) continue;
            float a[NEQ], b[NEQ];
#pragma unroll
            for (int m = 0; m < NEQ; m++) {
                a[m] = half(ql[m], h);
                b[m] = half(qr[m], h);
            }
            const Edge64 e = swe_edge64(gd, efix, a, b, trans);
#pragma unroll
            for (int m = 0; m < NEQ; m++) {
#pragma unroll
                for (int p = 0; p < NW; p++) half(W[p][m], h) = e.W[p][m];
                half(am[m], h) = e.am[m];
                half(ap[m], h) = e.ap[m];
                if (trans) {
                    half(Tm[m], h) = e.tm[m];
                    half(Tp[m], h) = e.tp[m];
                    half(Um[m], h) = e.um[m];
                    half(Up[m], h) = e.up[m];
                }
            }
#pragma unroll
            for (int p = 0; p < NW; p++) half(s[p], h) = e.s[p];
            half(L.u, h) = e.lin[0];
            half(L.v, h) = e.lin[1];
            half(L.c, h) = e.lin[2];
            half(L.r2c, h) = e.lin[3];
            (h ? bady : badx) = e.bad;
        }
    }

    template <int DIR>
    __device__ __forceinline__ void transverse(const Lin& L, const T* a, T* bm, T* bp) const
    {
        // eigenvectors of the direction 1 - DIR at the edge's Roe state: the
        // edge-tangential velocity L.v is the normal one there
        constexpr int vn = 2 - DIR, vt = 1 + DIR;
        const T u = L.v, v = L.u, c = L.c;
        const T b1 = ((u + c) * a[0] - a[vn]) * L.r2c;
        const T b2 = a[vt] - v * a[0];
        const T b3 = (a[vn] - (u - c) * a[0]) * L.r2c;
        const T l1 = u - c, l2 = u, l3 = u + c;
        // FP64 only: in FP32 (transverse option 2) the extra code measured
        // slower than the zero terms it saves
        if (sizeof(T) == 8 && l1 < T(0) && l3 > T(0)) {
            // subsonic across the split direction (the common case): B-
            // takes wave 1, B+ wave 3, the shear wave goes with the sign of
            // u; the same sums as below without their zero terms
            const T m1 = l1 * b1, p3 = l3 * b3;
            const T m2 = tmin0(l2) * b2, p2 = tmax0(l2) * b2;
            bm[0] = m1;
            bm[vn] = m1 * l1;
            bm[vt] = m1 * v + m2;
            bp[0] = p3;
            bp[vn] = p3 * l3;
            bp[vt] = p3 * v + p2;
            return;
        }
        const T m1 = tmin0(l1) * b1, m2 = tmin0(l2) * b2, m3 = tmin0(l3) * b3;
        const T p1 = tmax0(l1) * b1, p2 = tmax0(l2) * b2, p3 = tmax0(l3) * b3;
        bm[0] = m1 + m3;
        bm[vn] = m1 * (u - c) + m3 * (u + c);
        bm[vt] = (m1 + m3) * v + m2;
        bp[0] = p1 + p3;
        bp[vn] = p1 * (u - c) + p3 * (u + c);
        bp[vt] = (p1 + p3) * v + p2;
    }
};

// ---------------------------------------------------------------- Euler
template <typename T>
struct EulerRP {
    using real = T;
    static constexpr int NEQ = 4, NW = 3;
    static constexpr int NAUX = 0, NPLANE = NEQ;
    static constexpr bool POSITIVE = true;    // density rho > 0
    T gamma, gm1;
    bool efix;
    double gd, gm1d;  // gamma and gamma - 1 in FP64 (guarded edges)
    float gtau;       // FP32 guard threshold; negative: guard off
    struct Lin { T u, v, H, c, rc, gc2; };
    // every component of every wave can be non-zero
    template <int DIR>
    __host__ __device__ static constexpr bool wave_nz(int, int) { return true; }
    // the sweep keeps the limiter's dot products of the row below instead of
    // its 12 wave components (measured faster here)
    static constexpr bool CARRY_DOT = true;
    static constexpr bool PAIRED = sizeof(T) == 4;
    static constexpr bool SEEDED = false;   // no external pressure seed
    // max over the edge's waves of |s|: speeds u - c, u, u + c with c > 0
    __device__ __forceinline__ T max_speed(const Lin& L) const { return fabs(L.u) + L.c; }

    __device__ __forceinline__ void cell_speeds(const T* q, T& sx, T& sy) const
    {
        const T r1 = T(1) / q[0];
        const T u = q[1] * r1, v = q[2] * r1;
        const T p = gm1 * (q[3] - T(0.5) * q[0] * (u * u + v * v));
        const T c = sqrt(gamma * p * r1);
        sx = fabs(u) + c;
        sy = fabs(v) + c;
    }

    __host__ void setup(const double* param, int ef)
    {
        gamma = T(param[0]);
        gm1 = T(param[0] - 1.0);
        efix = ef != 0;
        gd = param[0];
        gm1d = param[0] - 1.0;
        gtau = param[3] == 0.0 ? GUARD_TAU_DEFAULT : float(param[3]);
    }
    __host__ __device__ __forceinline__ bool guard_on() const { return sizeof(T) == 4 && gtau >= 0.f; }
    // an edge the guard recomputes: across a near-vacuum front (the smaller
    // density below gtau times the larger; also for a density that is not a
    // positive number)
    __device__ __forceinline__ bool guarded(float rl, float rr) const
    {
        return !(rl >= gtau * rr) | !(rr >= gtau * rl);
    }
    // u_n + sgn c of a conserved state in FP64; false if not physical
    template <int DIR>
    __device__ __forceinline__ bool cspeed64(const T* q, double sgn, double& lam) const
    {
        constexpr int un = 1 + DIR, ut = 2 - DIR;
        const double r = q[0];
        if (!(r > 0.0)) return false;
        const double u = double(q[un]) / r, v = double(q[ut]) / r;
        const double p = gm1d * (double(q[3]) - 0.5 * r * (u * u + v * v));
        if (!(p > 0.0)) return false;
        lam = u + sgn * sqrt(gd * p / r);
        return true;
    }
    // Harten-Hyman for a wave with states qa on its left and qb on its
    // right, characteristic speed u + sgn c, Roe speed sroe: if both states
    // are physical and their speeds straddle zero, k = beta lam_a, beta =
    // (lam_b - sroe) / (lam_b - lam_a); otherwise k is left as it is.  F64:
    // the speeds and the split in FP64 (the guard's recompute of an FP32
    // step).
    // Returns true (FP32 form) when a speed lies within gtau times cref (the
    // Roe sound speed) of zero: a near-sonic edge for the FP64 guard.
    template <int DIR, bool F64 = false>
    __device__ __forceinline__ bool hh_fix(const T* qa, const T* qb, T sgn, T sroe, T cref, T& k) const
    {
        if constexpr (F64) {
            double la, lb;
            if (cspeed64<DIR>(qa, double(sgn), la) && cspeed64<DIR>(qb, double(sgn), lb) && la < 0.0 &&
                lb > 0.0)
                k = T((lb - double(sroe)) / (lb - la) * la);
            return false;
        } else {
            T la = T(0), lb = T(0);
            const bool ok = cspeed<DIR>(qa, sgn, la) && cspeed<DIR>(qb, sgn, lb);
            if (ok && la < T(0) && lb > T(0)) k = (lb - sroe) * rcp_(lb - la) * la;
            return ok && (fabs(la) < T(gtau) * cref || fabs(lb) < T(gtau) * cref);
        }
    }

    // speed u_n -+ c of a conserved state; false if not physical
    template <int DIR>
    __device__ __forceinline__ bool cspeed(const T* q, T sgn, T& lam) const
    {
        constexpr int un = 1 + DIR, ut = 2 - DIR;
        if (!(q[0] > T(0))) return false;
        T r1 = rcp_(q[0]);
        T u = q[un] * r1, v = q[ut] * r1;
        T p = gm1 * (q[3] - T(0.5) * q[0] * (u * u + v * v));
        if (!(p > T(0))) return false;
        lam = u + sgn * sqrt_(gamma * p * r1);
        return true;
    }

    // gamma (gamma - 1) rho^2 e of a state, with rho e = E - (m^2+n^2)/(2 rho)
    // (multiplied through by rho); positive iff the state is physical
    __device__ __forceinline__ T g_rho2e(const T* q) const
    {
        return gamma * gm1 * (q[3] * q[0] - T(0.5) * (q[1] * q[1] + q[2] * q[2]));
    }
    __device__ __forceinline__ f2 g_rho2e_pair(const f2* q) const
    {
        return p_mul(p_set(gamma * gm1),
                     p_fma(q[3], q[0], p_mul(p_set(-0.5f), p_fma(q[1], q[1], p_mul(q[2], q[2])))));
    }
    // u_n < c_K (sgn = false: u - c < 0) or u_n < -c (sgn = true: u + c < 0),
    // each also requiring a physical state
    template <int DIR>
    __device__ __forceinline__ bool slower_than_sound(const T* q, bool plus_side) const
    {
        constexpr int un = 1 + DIR;
        const T e = g_rho2e(q), m = q[un];
        if (!(q[0] > T(0) && e > T(0))) return false;
        // plus_side: u + c > 0 <=> m >= 0 or m^2 < e;  else: u - c < 0 <=> m <= 0 or m^2 < e
        return plus_side ? (m >= T(0) || m * m < e) : (m <= T(0) || m * m < e);
    }
    // u - c > 0 (plus_side = true) or u + c < 0 (plus_side = false)
    template <int DIR>
    __device__ __forceinline__ bool faster_than_sound(const T* q, bool plus_side) const
    {
        constexpr int un = 1 + DIR;
        const T e = g_rho2e(q), m = q[un];
        if (!(q[0] > T(0) && e > T(0))) return false;
        return plus_side ? (m > T(0) && m * m > e) : (m < T(0) && m * m > e);
    }

    template <int DIR>
    __device__ __forceinline__ void normal(const T* ql, const T* qr, T (&W)[NW][NEQ], T (&s)[NW],
                                           T* amdq, T* apdq, Lin& L, bool& bad) const
    {
        constexpr int un = 1 + DIR, ut = 2 - DIR;
        const T rl = ql[0], rr = qr[0];
        // sqrt(rho) weights from one reciprocal square root per state:
        // sqrt(rho) u = m / sqrt(rho), sqrt(rho) H = (E + p) / sqrt(rho)
        const T rsl = rsqrt_(rl), rsr = rsqrt_(rr);
        const T il = rsl * rsl, ir = rsr * rsr;
        const T kl = T(0.5) * (ql[un] * ql[un] + ql[ut] * ql[ut]) * il;
        const T kr = T(0.5) * (qr[un] * qr[un] + qr[ut] * qr[ut]) * ir;
        const T pl = gm1 * (ql[3] - kl), pr = gm1 * (qr[3] - kr);
        const T w = rcp_(rl * rsl + rr * rsr);
        const T u = (ql[un] * rsl + qr[un] * rsr) * w;
        const T v = (ql[ut] * rsl + qr[ut] * rsr) * w;
        const T H = ((ql[3] + pl) * rsl + (qr[3] + pr) * rsr) * w;
        const T c2 = gm1 * (H - T(0.5) * (u * u + v * v));
        // non-physical states are flagged; the arithmetic then yields NaNs
        bad = bad || !(rl > T(0) && rr > T(0) && c2 > T(0));
        const T rc = rsqrt_(c2);
        const T c = c2 * rc;
        const T gc2 = gm1 * rc * rc;
        const T d0 = qr[0] - ql[0], dn = qr[un] - ql[un], dt = qr[ut] - ql[ut], dE = qr[3] - ql[3];
        const T a_sh = dt - v * d0;
        const T a_en = gc2 * ((H - u * u - v * v) * d0 + u * dn + v * dt - dE);
        const T x = (dn - u * d0) * rc;
        const T a4 = T(0.5) * (d0 - a_en + x);
        const T a1 = T(0.5) * (d0 - a_en - x);
        W[0][0] = a1; W[0][un] = a1 * (u - c); W[0][ut] = a1 * v; W[0][3] = a1 * (H - u * c);
        W[1][0] = a_en; W[1][un] = a_en * u; W[1][ut] = a_en * v + a_sh;
        W[1][3] = a_en * T(0.5) * (u * u + v * v) + a_sh * v;
        W[2][0] = a4; W[2][un] = a4 * (u + c); W[2][ut] = a4 * v; W[2][3] = a4 * (H + u * c);
        s[0] = u - c;
        s[1] = u;
        s[2] = u + c;
        L.u = u; L.v = v; L.H = H; L.c = c; L.rc = rc; L.gc2 = gc2;

        T k0 = tmin0(s[0]), k2 = tmin0(s[2]);
        if (efix) {
            // Harten-Hyman, with the transonic test free of square roots and
            // divisions: for a state (rho, m, n, E) with rho e = rho E - (m^2 +
            // n^2)/2 > 0, u^2 < c^2 <=> m^2 < gamma (gamma-1) rho e.  The
            // speeds themselves are computed only for a transonic wave; an
            // intermediate state that is not physical leaves the wave unfixed.
            T qm[NEQ];
#pragma unroll
            for (int m = 0; m < NEQ; m++) qm[m] = ql[m] + W[0][m];
            // the intermediate state's test first: it rarely holds
            if (faster_than_sound<DIR>(qm, true) && slower_than_sound<DIR>(ql, false))
                hh_fix<DIR>(ql, qm, T(-1), s[0], c, k0);
#pragma unroll
            for (int m = 0; m < NEQ; m++) qm[m] = qr[m] - W[2][m];
            if (faster_than_sound<DIR>(qm, false) && slower_than_sound<DIR>(qr, true))
                hh_fix<DIR>(qm, qr, T(1), s[2], c, k2);
        }
        const T k1 = tmin0(s[1]);
#pragma unroll
        for (int m = 0; m < NEQ; m++) {
            amdq[m] = k0 * W[0][m] + k1 * W[1][m] + k2 * W[2][m];
            apdq[m] = s[0] * W[0][m] + s[1] * W[1][m] + s[2] * W[2][m] - amdq[m];
        }
    }

    template <int DIR>
    __device__ __forceinline__ void transverse(const Lin& L, const T* a, T* bm, T* bp) const
    {
        constexpr int vn = 2 - DIR, vt = 1 + DIR;
        const T u = L.v, v = L.u, c = L.c, H = L.H;   // u: normal to the split direction
        const T b_sh = a[vt] - v * a[0];
        const T b_en = L.gc2 * ((H - u * u - v * v) * a[0] + u * a[vn] + v * a[vt] - a[3]);
        const T x = (a[vn] - u * a[0]) * L.rc;
        const T b4 = T(0.5) * (a[0] - b_en + x);
        const T b1 = T(0.5) * (a[0] - b_en - x);
        const T l1 = u - c, l2 = u, l4 = u + c;
        const T ke = T(0.5) * (u * u + v * v);
        const T m1 = tmin0(l1) * b1, me = tmin0(l2) * b_en, ms = tmin0(l2) * b_sh, m4 = tmin0(l4) * b4;
        const T p1 = tmax0(l1) * b1, pe = tmax0(l2) * b_en, ps = tmax0(l2) * b_sh, p4 = tmax0(l4) * b4;
        bm[0] = m1 + me + m4;
        bm[vn] = m1 * (u - c) + me * u + m4 * (u + c);
        bm[vt] = (m1 + me + m4) * v + ms;
        bm[3] = m1 * (H - u * c) + me * ke + ms * v + m4 * (H + u * c);
        bp[0] = p1 + pe + p4;
        bp[vn] = p1 * (u - c) + pe * u + p4 * (u + c);
        bp[vt] = (p1 + pe + p4) * v + ps;
        bp[3] = p1 * (H - u * c) + pe * ke + ps * v + p4 * (H + u * c);
    }

    // ---- FP32 pairs: half .x an x-edge, .y a y-edge, both in the
    // edge-normal frame (component 1 normal, 2 tangential momentum); the
    // arithmetic of normal<0> / transverse<0>, two edges per instruction
    struct LinP { f2 u, v, H, c, rc, gc2; };
    // the scalar linearised state of half h (x-edge 0, y-edge 1)
    __device__ __forceinline__ Lin lin_half(const LinP& P, int h) const
    {
        return Lin{half(P.u, h), half(P.v, h), half(P.H, h), half(P.c, h), half(P.rc, h), half(P.gc2, h)};
    }
    __device__ __forceinline__ float max_speed(const LinP& L, int h) const
    {
        return fabs(half(L.u, h)) + half(L.c, h);
    }

    // hh: bit h set when half h met a near-sonic transonic wave (a speed
    // within gtau times the Roe sound speed of zero); F64FIX: the transonic
    // fix's speeds and split in FP64
    template <bool F64FIX = false>
    __device__ __forceinline__ void normal_pair(const f2* ql, const f2* qr, f2 (&W)[NW][NEQ],
                                                f2 (&s)[NW], f2* amdq, f2* apdq, LinP& L,
                                                bool& badx, bool& bady, int& hh) const
    {
        const f2 h2 = p_set(0.5f), g1 = p_set(gm1);
        const f2 rl = ql[0], rr = qr[0];
        const f2 rsl = p_rsqrt(rl), rsr = p_rsqrt(rr);
        const f2 il = p_mul(rsl, rsl), ir = p_mul(rsr, rsr);
        const f2 kl = p_mul(p_mul(h2, p_fma(ql[1], ql[1], p_mul(ql[2], ql[2]))), il);
        const f2 kr = p_mul(p_mul(h2, p_fma(qr[1], qr[1], p_mul(qr[2], qr[2]))), ir);
        const f2 pl = p_mul(g1, p_sub(ql[3], kl)), pr = p_mul(g1, p_sub(qr[3], kr));
        const f2 w = p_rcp(p_fma(rl, rsl, p_mul(rr, rsr)));
        const f2 u = p_mul(p_fma(ql[1], rsl, p_mul(qr[1], rsr)), w);
        const f2 v = p_mul(p_fma(ql[2], rsl, p_mul(qr[2], rsr)), w);
        const f2 H = p_mul(p_fma(p_add(ql[3], pl), rsl, p_mul(p_add(qr[3], pr), rsr)), w);
        const f2 q2 = p_fma(u, u, p_mul(v, v));
        const f2 c2 = p_mul(g1, p_fma(p_neg(h2), q2, H));
        badx = badx || !(rl.x > 0.f && rr.x > 0.f && c2.x > 0.f);
        bady = bady || !(rl.y > 0.f && rr.y > 0.f && c2.y > 0.f);
        const f2 rc = p_rsqrt(c2);
        const f2 c = p_mul(c2, rc);
        const f2 gc2 = p_mul(p_mul(g1, rc), rc);
        const f2 d0 = p_sub(qr[0], ql[0]), dn = p_sub(qr[1], ql[1]), dt = p_sub(qr[2], ql[2]);
        const f2 ndE = p_sub(ql[3], qr[3]);
        const f2 a_sh = p_fma(p_neg(v), d0, dt);
        // a_en = gc2 ((H - u^2 - v^2) d0 + u dn + v dt - dE)
        const f2 a_en = p_mul(gc2, p_fma(p_sub(H, q2), d0, p_fma(u, dn, p_fma(v, dt, ndE))));
        const f2 x = p_mul(p_fma(p_neg(u), d0, dn), rc);
        const f2 t = p_sub(d0, a_en);
        const f2 a4 = p_mul(h2, p_add(t, x)), a1 = p_mul(h2, p_sub(t, x));
        const f2 sm = p_sub(u, c), sp = p_add(u, c), uc = p_mul(u, c);
        W[0][0] = a1; W[0][1] = p_mul(a1, sm); W[0][2] = p_mul(a1, v); W[0][3] = p_mul(a1, p_sub(H, uc));
        W[1][0] = a_en; W[1][1] = p_mul(a_en, u); W[1][2] = p_fma(a_en, v, a_sh);
        W[1][3] = p_fma(p_mul(a_en, h2), q2, p_mul(a_sh, v));
        W[2][0] = a4; W[2][1] = p_mul(a4, sp); W[2][2] = p_mul(a4, v); W[2][3] = p_mul(a4, p_add(H, uc));
        s[0] = sm;
        s[1] = u;
        s[2] = sp;
        L.u = u; L.v = v; L.H = H; L.c = c; L.rc = rc; L.gc2 = gc2;

        f2 k0 = p_min0(sm), k2 = p_min0(sp);
        if (efix) {
            // the tests of normal() for both halves: for a state q, e = gamma
            // (gamma-1) rho^2 e_int, m its normal momentum; u < c <=> m <= 0 or
            // m^2 < e, u > c <=> m > 0 and m^2 > e, and the mirror tests for
            // u + c (each also needs rho > 0 and e > 0)
            f2 qm0[NEQ], qm2[NEQ];
#pragma unroll
            for (int m = 0; m < NEQ; m++) {
                qm0[m] = p_add(ql[m], W[0][m]);
                qm2[m] = p_sub(qr[m], W[2][m]);
            }
            // a wave can be transonic only if its middle state moves faster
            // than sound (rightward for the 1-wave, leftward for the 3-wave):
            // those tests come first, the outer states' only where one holds
            const f2 e_m0 = g_rho2e_pair(qm0), e_m2 = g_rho2e_pair(qm2);
            const f2 mm02 = p_mul(qm0[1], qm0[1]), mm22 = p_mul(qm2[1], qm2[1]);
            bool m_fast[2], m_neg[2];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const bool ok_m0 = (half(qm0[0], h) > 0.f) & (half(e_m0, h) > 0.f);
                const bool ok_m2 = (half(qm2[0], h) > 0.f) & (half(e_m2, h) > 0.f);
                // wave 1: u - c > 0 in the middle state; wave 3: u + c < 0 there
                m_fast[h] = ok_m0 & (half(qm0[1], h) > 0.f) & (half(mm02, h) > half(e_m0, h));
                m_neg[h] = ok_m2 & (half(qm2[1], h) < 0.f) & (half(mm22, h) > half(e_m2, h));
            }
            if (m_fast[0] | m_fast[1] | m_neg[0] | m_neg[1]) {
                const f2 e_l = g_rho2e_pair(ql), e_r = g_rho2e_pair(qr);
                const f2 ml2 = p_mul(ql[1], ql[1]), mr2 = p_mul(qr[1], qr[1]);
                bool t0[2], t2[2];
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const bool ok_l = (half(ql[0], h) > 0.f) & (half(e_l, h) > 0.f);
                    const bool ok_r = (half(qr[0], h) > 0.f) & (half(e_r, h) > 0.f);
                    // wave 1: u - c < 0 on the left; wave 3: u + c > 0 on the right
                    const bool l_slow = ok_l & ((half(ql[1], h) <= 0.f) | (half(ml2, h) < half(e_l, h)));
                    const bool r_pos = ok_r & ((half(qr[1], h) >= 0.f) | (half(mr2, h) < half(e_r, h)));
                    t0[h] = l_slow & m_fast[h];
                    t2[h] = m_neg[h] & r_pos;
                }
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    float qa[NEQ], qb[NEQ];
                    if (t0[h]) {
#pragma unroll
                        for (int m = 0; m < NEQ; m++) {
                            qa[m] = half(ql[m], h);
                            qb[m] = half(qm0[m], h);
                        }
                        if (hh_fix<0, F64FIX>(qa, qb, -1.f, half(sm, h), half(c, h), half(k0, h)))
                            hh |= 1 << h;
                    }
                    if (t2[h]) {
#pragma unroll
                        for (int m = 0; m < NEQ; m++) {
                            qa[m] = half(qm2[m], h);
                            qb[m] = half(qr[m], h);
                        }
                        if (hh_fix<0, F64FIX>(qa, qb, 1.f, half(sp, h), half(c, h), half(k2, h)))
                            hh |= 1 << h;
                    }
                }
            }
        }
        // A-dQ = sum_p k_p W^p, A+dQ = sum_p (s^p - k_p) W^p
        const f2 k1 = p_min0(u), j0 = p_sub(sm, k0), j1 = p_max0(u), j2 = p_sub(sp, k2);
#pragma unroll
        for (int m = 0; m < NEQ; m++) {
            amdq[m] = p_fma(k0, W[0][m], p_fma(k1, W[1][m], p_mul(k2, W[2][m])));
            apdq[m] = p_fma(j0, W[0][m], p_fma(j1, W[1][m], p_mul(j2, W[2][m])));
        }
    }

    template <bool SUB = true>   // the shallow-water form's flag; no subsonic form here
    __device__ __forceinline__ void transverse_pair(const LinP& L, const f2* a, f2* bm, f2* bp) const
    {
        // transverse<0> in the edge-normal frame: split direction normal
        // component 2, tangential 1
        const f2 h2 = p_set(0.5f);
        const f2 u = L.v, v = L.u, c = L.c, H = L.H;
        const f2 q2 = p_fma(u, u, p_mul(v, v));
        const f2 b_sh = p_fma(p_neg(v), a[0], a[1]);
        // b_en = gc2 ((H - u^2 - v^2) a0 + u a2 + v a1 - a3)
        const f2 b_en = p_mul(L.gc2, p_fma(p_sub(H, q2), a[0], p_fma(u, a[2], p_fma(v, a[1], p_neg(a[3])))));
        const f2 x = p_mul(p_fma(p_neg(u), a[0], a[2]), L.rc);
        const f2 t = p_sub(a[0], b_en);
        const f2 b4 = p_mul(h2, p_add(t, x)), b1 = p_mul(h2, p_sub(t, x));
        const f2 l1 = p_sub(u, c), l4 = p_add(u, c), uc = p_mul(u, c);
        const f2 ke = p_mul(h2, q2), e1 = p_sub(H, uc), e4 = p_add(H, uc);
        {
            const f2 n1 = p_min0(l1), n2 = p_min0(u), n4 = p_min0(l4);
            const f2 m1 = p_mul(n1, b1), me = p_mul(n2, b_en), ms = p_mul(n2, b_sh), m4 = p_mul(n4, b4);
            bm[0] = p_add(p_add(m1, me), m4);
            bm[2] = p_fma(m1, l1, p_fma(me, u, p_mul(m4, l4)));
            bm[1] = p_fma(bm[0], v, ms);
            bm[3] = p_fma(m1, e1, p_fma(me, ke, p_fma(ms, v, p_mul(m4, e4))));
        }
        {
            const f2 n1 = p_max0(l1), n2 = p_max0(u), n4 = p_max0(l4);
            const f2 m1 = p_mul(n1, b1), me = p_mul(n2, b_en), ms = p_mul(n2, b_sh), m4 = p_mul(n4, b4);
            bp[0] = p_add(p_add(m1, me), m4);
            bp[2] = p_fma(m1, l1, p_fma(me, u, p_mul(m4, l4)));
            bp[1] = p_fma(bp[0], v, ms);
            bp[3] = p_fma(m1, e1, p_fma(me, ke, p_fma(ms, v, p_mul(m4, e4))));
        }
    }

    // The FP64 guard of a pair: bit h set when half h is guarded.
    __device__ __forceinline__ int guard_mask(const f2* ql, const f2* qr, const LinP& L) const
    {
        if (!guard_on()) return 0;
        return int(guarded(ql[0].x, qr[0].x)) | (int(guarded(ql[0].y, qr[0].y)) << 1);
    }
    // Replaces the results of the guarded halves by their FP64 solve (and,
    // with trans, their FP64 transverse splits).
    __device__ __forceinline__ void guard_redo(const f2* ql, const f2* qr, int gm, bool trans,
                                               f2 (&W)[NW][NEQ], f2 (&s)[NW], f2* am, f2* ap,
                                               LinP& L, f2* Tm, f2* Tp, f2* Um, f2* Up, bool& badx,
                                               bool& bady) const
    {
#pragma unroll
        for (int h = 0; h < 2; h++) {
            if (!((gm >> h) & 1)) continue;
            float a[NEQ], b[NEQ];
#pragma unroll
            for (int m = 0; m < NEQ; m++) {
                a[m] = half(ql[m], h);
                b[m] = half(qr[m], h);
            }
            const Edge64 e = euler_edge64(gd, efix, a, b, trans);
#pragma unroll
            for (int m = 0; m < NEQ; m++) {
#pragma unroll
                for (int p = 0; p < NW; p++) half(W[p][m], h) = e.W[p][m];
                half(am[m], h) = e.am[m];
                half(ap[m], h) = e.ap[m];
                if (trans) {
                    half(Tm[m], h) = e.tm[m];
                    half(Tp[m], h) = e.tp[m];
                    half(Um[m], h) = e.um[m];
                    half(Up[m], h) = e.up[m];
                }
            }
#pragma unroll
            for (int p = 0; p < NW; p++) half(s[p], h) = e.s[p];
            half(L.u, h) = e.lin[0];
            half(L.v, h) = e.lin[1];
            half(L.H, h) = e.lin[2];
            half(L.c, h) = e.lin[3];
            half(L.rc, h) = e.lin[4];
            half(L.gc2, h) = e.lin[5];
            (h ? bady : badx) = !(a[0] > 0.f && b[0] > 0.f) || e.bad;
        }
    }
};

// ---------------------------------------------------------------- FP64 guard: edge solves
static __device__ __forceinline__ Edge64 swe_edge64(double g, bool efix, const float (&a)[3],
                                                 const float (&b)[3], bool trans)
{
    SweRP<double> r;
    r.g = g;
    r.gd = g;
    r.efix = efix;
    r.gtau = -1.f;
    double ql[3], qr[3], W[3][3], s[3], am[3], ap[3];
#pragma unroll
    for (int m = 0; m < 3; m++) {
        ql[m] = a[m];
        qr[m] = b[m];
    }
    typename SweRP<double>::Lin L;
    bool bad = false;
    r.template normal<0>(ql, qr, W, s, am, ap, L, bad);
    Edge64 e{};
#pragma unroll
    for (int m = 0; m < 3; m++) {
#pragma unroll
        for (int p = 0; p < 3; p++) e.W[p][m] = float(W[p][m]);
        e.am[m] = float(am[m]);
        e.ap[m] = float(ap[m]);
    }
#pragma unroll
    for (int p = 0; p < 3; p++) e.s[p] = float(s[p]);
    e.lin[0] = float(L.u); e.lin[1] = float(L.v); e.lin[2] = float(L.c); e.lin[3] = float(L.r2c);
    if (trans) {
        double t1[3], t2[3];
        r.template transverse<0>(L, am, t1, t2);
#pragma unroll
        for (int m = 0; m < 3; m++) { e.tm[m] = float(t1[m]); e.tp[m] = float(t2[m]); }
        r.template transverse<0>(L, ap, t1, t2);
#pragma unroll
        for (int m = 0; m < 3; m++) { e.um[m] = float(t1[m]); e.up[m] = float(t2[m]); }
    }
    e.bad = bad;
    return e;
}

static __device__ __forceinline__ Edge64 euler_edge64(double gamma, bool efix, const float (&a)[4],
                                                   const float (&b)[4], bool trans)
{
    EulerRP<double> r;
    r.gamma = gamma;
    r.gm1 = gamma - 1.0;
    r.gd = gamma;
    r.gm1d = gamma - 1.0;
    r.efix = efix;
    r.gtau = -1.f;
    double ql[4], qr[4], W[3][4], s[3], am[4], ap[4];
#pragma unroll
    for (int m = 0; m < 4; m++) {
        ql[m] = a[m];
        qr[m] = b[m];
    }
    typename EulerRP<double>::Lin L;
    bool bad = false;
    r.template normal<0>(ql, qr, W, s, am, ap, L, bad);
    Edge64 e{};
#pragma unroll
    for (int m = 0; m < 4; m++) {
#pragma unroll
        for (int p = 0; p < 3; p++) e.W[p][m] = float(W[p][m]);
        e.am[m] = float(am[m]);
        e.ap[m] = float(ap[m]);
    }
#pragma unroll
    for (int p = 0; p < 3; p++) e.s[p] = float(s[p]);
    e.lin[0] = float(L.u); e.lin[1] = float(L.v); e.lin[2] = float(L.H);
    e.lin[3] = float(L.c); e.lin[4] = float(L.rc); e.lin[5] = float(L.gc2);
    if (trans) {
        double t1[4], t2[4];
        r.template transverse<0>(L, am, t1, t2);
#pragma unroll
        for (int m = 0; m < 4; m++) { e.tm[m] = float(t1[m]); e.tp[m] = float(t2[m]); }
        r.template transverse<0>(L, ap, t1, t2);
#pragma unroll
        for (int m = 0; m < 4; m++) { e.um[m] = float(t1[m]); e.up[m] = float(t2[m]); }
    }
    e.bad = bad;
    return e;
}

// ---------------------------------------------------------------- Euler, exact solution
// Godunov normal solve: the exact Riemann solution of the normal problem
// (Toro ch. 4; p* by Newton from Toro's adaptive PV/TR/TS guess) gives the
// fluctuations as flux differences to the state at x/t = 0 (Toro §4.5), and
// the waves as the jumps across the two nonlinear waves and the contact (the
// tangential velocity jumps with the contact), at the shock speeds or the
// rarefaction heads and u*.  The transverse split is Roe's at the edge's Roe
// average (EulerRP::transverse).  No entropy fix is needed.
template <typename T>
struct EulerGodunovRP : EulerRP<T> {
    using Base = EulerRP<T>;
    using real = T;
    using Base::NEQ;
    using Base::NW;
    using Base::gamma;
    using Base::gm1;
    static constexpr bool PAIRED = false;   // scalar solves only
    // accepts a pressure seed for Newton (normal_seeded), e.g. the learned one
    static constexpr bool SEEDED = true;
    static constexpr bool CARRY_DOT = true;
    struct Lin : Base::Lin { T smax; };
    // gamma's constants, set once on the host (no divisions in the solve):
    // z = (g-1)/(2g), g6 = (g-1)/(g+1), a2 = 2/(g+1), sk = (g+1)/(2g),
    // ig = 1/g, igm1 = 1/(g-1), tgm1 = 2/(g-1), rz = 1/z
    T z, g6, a2, sk, ig, igm1, tgm1, rz;
    __host__ void setup(const double* param, int ef)
    {
        Base::setup(param, ef);
        const double g = param[0];
        z = T(0.5 * (g - 1.0) / g);
        g6 = T((g - 1.0) / (g + 1.0));
        a2 = T(2.0 / (g + 1.0));
        sk = T((g + 1.0) / (2.0 * g));
        ig = T(1.0 / g);
        igm1 = T(1.0 / (g - 1.0));
        tgm1 = T(2.0 / (g - 1.0));
        rz = T(2.0 * g / (g - 1.0));
    }

    // primitive (rho, u_n, u_t, p) and sound speed of a state on an edge of
    // normal DIR
    template <int DIR>
    __device__ __forceinline__ void prim(const T* q, T& r, T& un, T& ut, T& p, T& c) const
    {
        r = q[0];
        const T ir = rcp_(r);
        un = q[1 + DIR] * ir;
        ut = q[2 - DIR] * ir;
        p = gm1 * (q[3] - T(0.5) * r * (un * un + ut * ut));
        c = sqrt_(gamma * p * ir);
    }
    // a mild jump: p_max < 2 p_min, the pressure-ratio part of Toro's
    // adaptive rule.  There the PV or TR/TS guess already lies close to p*,
    // and the network is not consulted.  (Kinetic energy (m_1^2 + m_2^2) /
    // (2 rho) does not depend on the edge's direction.)
    __device__ __forceinline__ bool seed_mild(const T* ql, const T* qr) const
    {
        const T pl = gm1 * (ql[3] - T(0.5) * (ql[1] * ql[1] + ql[2] * ql[2]) * rcp_(ql[0]));
        const T pr = gm1 * (qr[3] - T(0.5) * (qr[1] * qr[1] + qr[2] * qr[2]) * rcp_(qr[0]));
        return fmax(pl, pr) < T(2) * fmin(pl, pr);
    }
    // the seed network's ten raw inputs of the edge's normal problem (ln rho,
    // ln p, ln c of both sides, du, du/(c_L + c_R), ln p_TR, ln max(p_PV,
    // 1e-6)) and the two-rarefaction guess p_TR its output multiplies
    template <int DIR>
    __device__ __forceinline__ void seed_features(const T* ql, const T* qr, float (&x)[10], float& ptr) const
    {
        T rl, ul, vl, pl, cl, rr, ur, vr, pr, cr;
        prim<DIR>(ql, rl, ul, vl, pl, cl);
        prim<DIR>(qr, rr, ur, vr, pr, cr);
        const T du = ur - ul;
        const T pv = T(0.5) * (pl + pr) - T(0.125) * du * (rl + rr) * (cl + cr);
        const T tr = pow_((cl + cr - T(0.5) * gm1 * du) * rcp_(cl * pow_(pl, -z) + cr * pow_(pr, -z)), rz);
        x[0] = __logf(float(rl));
        x[1] = __logf(float(rr));
        x[2] = __logf(float(pl));
        x[3] = __logf(float(pr));
        x[4] = __logf(float(cl));
        x[5] = __logf(float(cr));
        x[6] = float(du);
        x[7] = float(du * rcp_(cl + cr));
        x[8] = __logf(float(tr));
        x[9] = __logf(fmaxf(float(pv), 1e-6f));
        ptr = float(tr);
    }
    __device__ __forceinline__ T max_speed(const Lin& L) const { return L.smax; }

    // one side's branch of the pressure function f_K(p) and f_K'(p)
    __device__ __forceinline__ void fK(T p, T rK, T pK, T cK, T& f, T& fd) const
    {
        if (p > pK) {
            const T A = a2 * rcp_(rK), B = g6 * pK;
            const T q = sqrt_(A * rcp_(B + p));
            f = (p - pK) * q;
            fd = q * (T(1) - T(0.5) * (p - pK) * rcp_(B + p));
        } else {
            const T r = p * rcp_(pK);
            const T pz = pow_(r, z);
            f = tgm1 * cK * (pz - T(1));
            fd = pz * rcp_(r * rK * cK);   // (p/p_K)^(-(gamma+1)/(2 gamma)) / (rho_K c_K)
        }
    }
    __device__ __forceinline__ T star_density(T rK, T pK, T ps) const
    {
        const T r = ps * rcp_(pK);
        if (ps > pK) {
            return rK * (r + g6) * rcp_(g6 * r + T(1));
        }
        return rK * pow_(r, ig);
    }
    __device__ __forceinline__ T shock_speed(T uK, T pK, T cK, T ps, T sgn) const
    {
        return uK + sgn * cK * sqrt_(sk * ps * rcp_(pK) + z);
    }
    // normal flux of (rho, u_n, u_t, p) in the edge frame (0: mass, 1: normal
    // momentum, 2: tangential momentum, 3: energy)
    __device__ __forceinline__ void nflux(T rho, T un, T ut, T p, T* f) const
    {
        const T E = p * igm1 + T(0.5) * rho * (un * un + ut * ut);
        f[0] = rho * un;
        f[1] = rho * un * un + p;
        f[2] = rho * un * ut;
        f[3] = un * (E + p);
    }
    __device__ __forceinline__ void cons(T rho, T un, T ut, T p, T* q) const
    {
        q[0] = rho;
        q[1] = rho * un;
        q[2] = rho * ut;
        q[3] = p * igm1 + T(0.5) * rho * (un * un + ut * ut);
    }

    template <int DIR>
    __device__ __forceinline__ void normal(const T* ql, const T* qr, T (&W)[NW][NEQ], T (&s)[NW],
                                           T* amdq, T* apdq, Lin& L, bool& bad) const
    {
        (void)normal_seeded<DIR>(ql, qr, T(0), W, s, amdq, apdq, L, bad);
    }

    // The normal solve with Newton started from pseed when it is a plausible
    // pressure (finite, within [1e-6 p_min, 1e6 p_max]), else from Toro's
    // adaptive guess; a seeded run that does not converge restarts from that
    // guess.  Returns the number of Newton updates.
    template <int DIR>
    __device__ __forceinline__ int normal_seeded(const T* ql, const T* qr, T pseed, T (&W)[NW][NEQ],
                                                 T (&s)[NW], T* amdq, T* apdq, Lin& L, bool& bad) const
    {
        constexpr int un_ = 1 + DIR, ut_ = 2 - DIR;
        // Roe average of the edge, for the transverse split and as a guard
        const T rl = ql[0], rr = qr[0];
        const T rsl = rsqrt_(rl), rsr = rsqrt_(rr);
        const T il = rsl * rsl, ir = rsr * rsr;
        const T ul = ql[un_] * il, vl = ql[ut_] * il, ur = qr[un_] * ir, vr = qr[ut_] * ir;
        const T pl = gm1 * (ql[3] - T(0.5) * rl * (ul * ul + vl * vl));
        const T pr = gm1 * (qr[3] - T(0.5) * rr * (ur * ur + vr * vr));
        const T w = rcp_(rl * rsl + rr * rsr);
        L.u = (ql[un_] * rsl + qr[un_] * rsr) * w;
        L.v = (ql[ut_] * rsl + qr[ut_] * rsr) * w;
        L.H = ((ql[3] + pl) * rsl + (qr[3] + pr) * rsr) * w;
        const T c2 = gm1 * (L.H - T(0.5) * (L.u * L.u + L.v * L.v));
        L.rc = rsqrt_(c2);
        L.c = c2 * L.rc;
        L.gc2 = gm1 * L.rc * L.rc;
        const T cl = sqrt_(gamma * pl * il), cr = sqrt_(gamma * pr * ir);
        const bool phys = rl > T(0) && rr > T(0) && pl > T(0) && pr > T(0) && c2 > T(0);
        // vacuum is generated when 2 (c_L + c_R)/(gamma - 1) <= u_R - u_L
        const bool vac = T(2) * (cl + cr) <= gm1 * (ur - ul);
        bad = bad || !phys || vac;

        // star pressure: Newton on f_L + f_R + u_R - u_L from the adaptive guess
        const T du = ur - ul;
        const T pmin = fmin(pl, pr), pmax = fmax(pl, pr);
        T ppv = T(0.5) * (pl + pr) - T(0.125) * du * (rl + rr) * (cl + cr);
        ppv = fmax(ppv, pmin * T(1e-6));
        T p0;
        if (pmax < T(2) * pmin && ppv >= pmin && ppv <= pmax) {
            p0 = ppv;
        } else if (ppv < pmin) {
            p0 = pow_((cl + cr - T(0.5) * gm1 * du) * rcp_(cl * pow_(pl, -z) + cr * pow_(pr, -z)), rz);
        } else {
            const T gl = sqrt_(a2 * rcp_(rl * (g6 * pl + ppv)));
            const T gr = sqrt_(a2 * rcp_(rr * (g6 * pr + ppv)));
            p0 = (gl * pl + gr * pr - du) * rcp_(gl + gr);
        }
        const T tol = sizeof(T) == 4 ? T(1e-6) : T(1e-14);
        const bool seeded = pseed >= T(1e-6) * pmin && pseed <= T(1e6) * pmax;   // false for NaN
        T ps = seeded ? pseed : fmax(p0, pmin * T(1e-6));
        int updates = 0;
        // branch values and slopes at the last iterate pprev, kept for u*
        T fl = T(0), fdl = T(0), fr = T(0), fdr = T(0), pprev = ps;
        for (int pass = seeded ? 0 : 1; pass < 2; pass++) {
            bool conv = false;
            for (int it = 0; it < 40; it++) {
                fK(ps, rl, pl, cl, fl, fdl);
                fK(ps, rr, pr, cr, fr, fdr);
                pprev = ps;
                T pn = ps - (fl + fr + du) * rcp_(fdl + fdr);
                pn = fmax(pn, pmin * T(1e-8));
                updates++;
                conv = fabs(pn - ps) <= tol * pn;
                ps = pn;
                if (conv || !(ps == ps)) break;
            }
            if (conv) break;
            if (pass == 0) ps = fmax(p0, pmin * T(1e-6));   // the seeded run failed: restart from the guess
        }
        // u* = (u_l + u_r)/2 + (f_R(p*) - f_L(p*))/2 (Toro, ch. 4), with the
        // branches taken at p* to first order from the last iterate: the
        // final step moved p by at most tol p, so the neglected term is of
        // order (tol p)^2 and two more branch evaluations are saved
        const T us = T(0.5) * (ul + ur) + T(0.5) * ((fr - fl) + (fdr - fdl) * (ps - pprev));

        // waves and speeds, in the edge frame, then to the physical frame
        T qL[4], qSL[4], qSR[4], qR[4];
        cons(rl, ul, vl, pl, qL);
        cons(star_density(rl, pl, ps), us, vl, ps, qSL);
        cons(star_density(rr, pr, ps), us, vr, ps, qSR);
        cons(rr, ur, vr, pr, qR);
        const int fc[4] = {0, un_, ut_, 3};
#pragma unroll
        for (int m = 0; m < 4; m++) {
            W[0][fc[m]] = qSL[m] - qL[m];
            W[1][fc[m]] = qSR[m] - qSL[m];
            W[2][fc[m]] = qR[m] - qSR[m];
        }
        s[0] = ps > pl ? shock_speed(ul, pl, cl, ps, T(-1)) : ul - cl;
        s[1] = us;
        s[2] = ps > pr ? shock_speed(ur, pr, cr, ps, T(1)) : ur + cr;
        L.smax = fmax(fmax(fabs(s[0]), fabs(s[2])), fabs(s[1]));

        // the state at x/t = 0 (Toro §4.5): on the side of the contact that
        // holds the interface, behind or ahead of that side's wave, or inside
        // its fan at the sonic point
        const bool left = us >= T(0);
        const T rK = left ? rl : rr, pK = left ? pl : pr, uK = left ? ul : ur, cK = left ? cl : cr;
        const T vK = left ? vl : vr, sgn = left ? T(-1) : T(1);
        T r0, u0, p0s;
        if (ps > pK) {
            const T S = shock_speed(uK, pK, cK, ps, sgn);
            const bool ahead = left ? S >= T(0) : S <= T(0);
            r0 = ahead ? rK : star_density(rK, pK, ps);
            u0 = ahead ? uK : us;
            p0s = ahead ? pK : ps;
        } else {
            const T head = uK + sgn * cK;
            const T cs = cK * pow_(ps * rcp_(pK), z);
            const T tail = us + sgn * cs;
            if (left ? head >= T(0) : head <= T(0)) {
                r0 = rK; u0 = uK; p0s = pK;
            } else if (left ? tail <= T(0) : tail >= T(0)) {
                r0 = star_density(rK, pK, ps); u0 = us; p0s = ps;
            } else {
                const T c = a2 * (cK - sgn * T(0.5) * gm1 * uK);
                const T rc_ = c * rcp_(cK);
                u0 = -sgn * c;
                r0 = rK * pow_(rc_, tgm1);
                p0s = pK * pow_(rc_, gamma * tgm1);
            }
        }
        T f0[4], fL[4], fR[4];
        nflux(r0, u0, vK, p0s, f0);
        nflux(rl, ul, vl, pl, fL);
        nflux(rr, ur, vr, pr, fR);
#pragma unroll
        for (int m = 0; m < 4; m++) {
            amdq[fc[m]] = f0[m] - fL[m];
            apdq[fc[m]] = fR[m] - f0[m];
        }
        return updates;
    }
};

}  // namespace mc
