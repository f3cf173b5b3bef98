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
// inside the FP32 parity tolerance); FP64 keeps correctly rounded division
// and square root.
__device__ __forceinline__ float rcp_(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double rcp_(double x) { return 1.0 / x; }
__device__ __forceinline__ float rsqrt_(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double rsqrt_(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float sqrt_(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }

// ---------------------------------------------------------------- acoustics
template <typename T>
struct AcousticsRP {
    using real = T;
    static constexpr int NEQ = 3, NW = 2;
    static constexpr bool POSITIVE = false;   // no positivity constraint on (p, u, v)
    T c, Z, inv2Z;
    bool efix;  // unused: linear system
    struct Lin {};
    // component m of wave p can be non-zero (the tangential velocity never is)
    template <int DIR>
    __host__ __device__ static constexpr bool wave_nz(int, int m) { return m != 2 - DIR; }
    // the sweep keeps the y-edge waves of the row below (not their products)
    static constexpr bool CARRY_DOT = false;

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

// ---------------------------------------------------------------- shallow water
template <typename T>
struct SweRP {
    using real = T;
    static constexpr int NEQ = 3, NW = 3;
    static constexpr bool POSITIVE = true;    // depth h > 0
    T g;
    bool efix;
    struct Lin { T u, v, c, r2c; };
    // component m of wave p can be non-zero: the shear wave moves only the
    // tangential momentum
    template <int DIR>
    __host__ __device__ static constexpr bool wave_nz(int p, int m) { return p != 1 || m == 2 - DIR; }
    // the sweep keeps the y-edge waves of the row below (measured faster here)
    static constexpr bool CARRY_DOT = false;
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
    }

    template <int DIR>
    __device__ __forceinline__ void normal(const T* ql, const T* qr, T (&W)[NW][NEQ], T (&s)[NW],
                                           T* amdq, T* apdq, Lin& L, bool& bad) const
    {
        constexpr int un = 1 + DIR, ut = 2 - DIR;
        const T hl = ql[0], hr = qr[0];
        // a non-positive depth is flagged; the arithmetic then yields NaNs,
        // which the caller's status word reports
        bad = bad || !(hl > T(0) && hr > T(0));
        // Roe average: sqrt(h) u = hu / sqrt(h), so one reciprocal square
        // root per state gives both weights
        const T rsl = rsqrt_(hl), rsr = rsqrt_(hr);
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
            const T hul = ql[un], hum = ql[un] + W[0][un], hm = hl + W[0][0];
            const bool l_neg = hul <= T(0) || hul * hul < g * hl * hl * hl;
            const bool r_pos = hm > T(0) && hum > T(0) && hum * hum > g * hm * hm * hm;
            if (l_neg && r_pos) {
                const T lam_l = hul * rcp_(hl) - sqrt_(g * hl);
                const T lam_r = hum * rcp_(hm) - sqrt_(g * hm);
                if (lam_l < T(0) && lam_r > T(0)) k0 = (lam_r - s[0]) * rcp_(lam_r - lam_l) * lam_l;
            }
            const T hur = qr[un], hun = qr[un] - W[2][un], hn = hr - W[2][0];
            const bool n_neg = hn > T(0) && hun < T(0) && hun * hun > g * hn * hn * hn;
            const bool rr_pos = hur >= T(0) || hur * hur < g * hr * hr * hr;
            if (n_neg && rr_pos) {
                const T ll = hun * rcp_(hn) + sqrt_(g * hn);
                const T lr = hur * rcp_(hr) + sqrt_(g * hr);
                if (ll < T(0) && lr > T(0)) k2 = (lr - s[2]) * rcp_(lr - ll) * ll;
            }
        }
        // A-dQ = sum_p k_p W^p, A+dQ = sum_p (s^p - k_p) W^p (k_p = min(s^p, 0)
        // unless the entropy fix replaced it), over the non-zero components
        const T k1 = tmin0(s[1]);
        const T m1 = k0 * a1, m2 = k1 * a2, m3 = k2 * a3;
        const T p1 = (s[0] - k0) * a1, p2 = (s[1] - k1) * a2, p3 = (s[2] - k2) * a3;
        amdq[0] = m1 + m3;
        amdq[un] = m1 * (u - c) + m3 * (u + c);
        amdq[ut] = (m1 + m3) * v + m2;
        apdq[0] = p1 + p3;
        apdq[un] = p1 * (u - c) + p3 * (u + c);
        apdq[ut] = (p1 + p3) * v + p2;
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
    static constexpr bool POSITIVE = true;    // density rho > 0
    T gamma, gm1;
    bool efix;
    struct Lin { T u, v, H, c, rc, gc2; };
    // every component of every wave can be non-zero
    template <int DIR>
    __host__ __device__ static constexpr bool wave_nz(int, int) { return true; }
    // the sweep keeps the limiter's dot products of the row below instead of
    // its 12 wave components (measured faster here)
    static constexpr bool CARRY_DOT = true;
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
            if (slower_than_sound<DIR>(ql, false) && faster_than_sound<DIR>(qm, true)) {
                T ll, lr;
                if (cspeed<DIR>(ql, T(-1), ll) && cspeed<DIR>(qm, T(-1), lr) && ll < T(0) &&
                    lr > T(0))
                    k0 = (lr - s[0]) * rcp_(lr - ll) * ll;
            }
#pragma unroll
            for (int m = 0; m < NEQ; m++) qm[m] = qr[m] - W[2][m];
            if (faster_than_sound<DIR>(qm, false) && slower_than_sound<DIR>(qr, true)) {
                T ll, lr;
                if (cspeed<DIR>(qm, T(1), ll) && cspeed<DIR>(qr, T(1), lr) && ll < T(0) &&
                    lr > T(0))
                    k2 = (lr - s[2]) * rcp_(lr - ll) * ll;
            }
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
};

}  // namespace mc
