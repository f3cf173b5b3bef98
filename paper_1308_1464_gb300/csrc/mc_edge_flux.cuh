// mc_edge_flux.cuh -- the flux through one edge under the wave-propagation
// step, evaluated pointwise from the state around the edge.
//
// With a conservative normal solve (A-dQ + A+dQ = f(Q_high) - f(Q_low)) the
// step's update of a cell is minus the difference of its edges' fluxes
//
//   F = f(Q_low) + A-dQ + F~,
//
// F~ the limited correction sum 1/2 |s| (1 - dt/d |s|) phi(theta) W and the
// transverse terms: the fluctuations entering the edge's two cells across
// the edges of the other direction, split along the edge normal, the high
// cell giving its part that moves to lower indices and the low cell its part
// that moves to higher ones, each times -dt/(2 d_other) (LeVeque 2002, §6.14
// and ch. 21).  Transverse option 2 splits those edges' fluctuations with
// their limited corrections (A+dQ - F~ into the high cell, A-dQ + F~ into the
// low one).  The refined-patch coupling needs this flux at the edges on the
// patches' boundaries, where the fused step keeps nothing.
#pragma once

#include "mc_sweep.cuh"

namespace mc {

// ---- physical flux along direction DIR of a conserved state

template <int DIR, typename T>
__device__ __forceinline__ void phys_flux(const AcousticsRP<T>& rp, const T* q, T* f)
{
    // p_t + K div u = 0, u_t + grad p / rho = 0 with K = Z c, 1/rho = c / Z
    f[0] = rp.Z * rp.c * q[1 + DIR];
    f[1 + DIR] = q[0] * rp.c / rp.Z;
    f[2 - DIR] = T(0);
}

template <int DIR, typename T>
__device__ __forceinline__ void phys_flux(const AdvectionRP<T>& rp, const T* q, T* f)
{
    f[0] = (DIR == 0 ? rp.u : rp.v) * q[0];
}

template <int DIR, typename T>
__device__ __forceinline__ void phys_flux(const SweRP<T>& rp, const T* q, T* f)
{
    constexpr int un = 1 + DIR, ut = 2 - DIR;
    const T u = q[un] / q[0];
    f[0] = q[un];
    f[un] = q[un] * u + T(0.5) * rp.g * q[0] * q[0];
    f[ut] = q[ut] * u;
}

template <int DIR, typename T>
__device__ __forceinline__ void phys_flux(const EulerRP<T>& rp, const T* q, T* f)
{
    constexpr int un = 1 + DIR, ut = 2 - DIR;
    const T u = q[un] / q[0], v = q[ut] / q[0];
    const T p = rp.gm1 * (q[3] - T(0.5) * q[0] * (u * u + v * v));
    f[0] = q[un];
    f[un] = q[un] * u + p;
    f[ut] = q[ut] * u;
    f[3] = (q[3] + p) * u;
}

// A state array in the library layout: plane m of cell (i, j) at
// q[m ld_field + (j + 2) ld_x + x_offset + i].
template <typename T>
struct StateView {
    const T* q;
    long long ld_x, ld_field, x_offset;
    template <int NP>
    __device__ __forceinline__ void cell(int i, int j, T (&v)[NP]) const
    {
        const T* c = q + (long long)(j + 2) * ld_x + x_offset + i;
#pragma unroll
        for (int m = 0; m < NP; m++) v[m] = c[m * ld_field];
    }
};

struct EdgeScheme {
    int limiter;
    bool second;
    int transverse;   // 0, 1, 2 (2 acts as 1 at first order)
};

// The cells around an edge of normal DIR in (along, across) offsets from its
// high cell: along a = -1 is the low cell, a = 0 the high cell.
template <int DIR, typename T, int NP>
__device__ __forceinline__ void around(const StateView<T>& V, int i, int j, int a, int b, T (&v)[NP])
{
    if (DIR == 0) V.template cell<NP>(i + a, j + b, v);
    else V.template cell<NP>(i + b, j + a, v);
}

// normal solve of direction D between cells lo and hi (a call, not inlined:
// an edge flux needs up to 19 of them)
template <class RP, int D>
__device__ __noinline__ void solve_pair(const RP& rp, const typename RP::real* lo,
                                        const typename RP::real* hi,
                                        typename RP::real (&W)[RP::NW][RP::NEQ],
                                        typename RP::real (&s)[RP::NW], typename RP::real* am,
                                        typename RP::real* ap, typename RP::Lin& L)
{
    bool bad = false;
    rp.template normal<D>(lo, hi, W, s, am, ap, L, bad);
}

// Limited correction of the edge of normal D whose three cells below it and
// two above along D are c0 .. c3 (c1 | c2 the edge itself, c0 | c1 and
// c2 | c3 its neighbours).
template <class RP, int D>
__device__ __forceinline__ void correction4(const RP& rp, const typename RP::real* c0,
                                            const typename RP::real* c1,
                                            const typename RP::real* c2,
                                            const typename RP::real* c3, typename RP::real dtd,
                                            int limiter, typename RP::real* out)
{
    using T = typename RP::real;
    constexpr int N = RP::NEQ, NW = RP::NW;
    T W0[NW][N], Wl[NW][N], Wh[NW][N], s0[NW], sl[NW], sh[NW], am[N], ap[N];
    typename RP::Lin L;
    solve_pair<RP, D>(rp, c1, c2, W0, s0, am, ap, L);
    solve_pair<RP, D>(rp, c0, c1, Wl, sl, am, ap, L);
    solve_pair<RP, D>(rp, c2, c3, Wh, sh, am, ap, L);
    T th[NW], phi[NW];
#pragma unroll
    for (int p = 0; p < NW; p++) {
        T dl = T(0), dr = T(0);
#pragma unroll
        for (int m = 0; m < N; m++) {
            const T wu = s0[p] > T(0) ? Wl[p][m] : Wh[p][m];
            dl += wu * W0[p][m];
            dr += W0[p][m] * W0[p][m];
        }
        th[p] = dl * rcp_(dr);
    }
    limiter_phis<NW>(limiter, th, phi);
#pragma unroll
    for (int m = 0; m < N; m++) out[m] = T(0);
#pragma unroll
    for (int p = 0; p < NW; p++) {
        const T as = fabs(s0[p]);
        const T cf = T(0.5) * as * (T(1) - dtd * as) * phi[p];
#pragma unroll
        for (int m = 0; m < N; m++) out[m] += cf * W0[p][m];
    }
}

// The flux F through the edge of normal DIR with high cell (i, j); dtd =
// dt / d along DIR, dto = dt / d across.
template <class RP, int DIR>
__device__ void edge_flux(const RP& rp, const StateView<typename RP::real>& V, int i, int j,
                          typename RP::real dtd, typename RP::real dto, const EdgeScheme& S,
                          typename RP::real* F)
{
    using T = typename RP::real;
    constexpr int N = RP::NEQ, NW = RP::NW, NP = RP::NPLANE, O = 1 - DIR;
    T cm2[NP], cm1[NP], c0[NP], cp1[NP];
    around<DIR>(V, i, j, -2, 0, cm2);
    around<DIR>(V, i, j, -1, 0, cm1);
    around<DIR>(V, i, j, 0, 0, c0);
    around<DIR>(V, i, j, 1, 0, cp1);
    {
        T W[NW][N], s[NW], am[N], ap[N];
        typename RP::Lin L;
        solve_pair<RP, DIR>(rp, cm1, c0, W, s, am, ap, L);
        phys_flux<DIR>(rp, cm1, F);
#pragma unroll
        for (int m = 0; m < N; m++) F[m] += am[m];
    }
    if (S.second) {
        T c[N];
        correction4<RP, DIR>(rp, cm2, cm1, c0, cp1, dtd, S.limiter, c);
#pragma unroll
        for (int m = 0; m < N; m++) F[m] += c[m];
    }
    if (S.transverse == 0) return;
    const bool t2 = S.transverse == 2 && S.second;
    // the two cells of the edge (side 0 low, 1 high) and the edges of
    // normal O below (e = 0) and above (e = 1) each of them
#pragma unroll
    for (int side = 0; side < 2; side++) {
        const int a = side - 1;
        T b2[NP], b1[NP], bc[NP], bp1[NP], bp2[NP];
        around<DIR>(V, i, j, a, -2, b2);
        around<DIR>(V, i, j, a, -1, b1);
        around<DIR>(V, i, j, a, 0, bc);
        around<DIR>(V, i, j, a, 1, bp1);
        around<DIR>(V, i, j, a, 2, bp2);
#pragma unroll
        for (int e = 0; e < 2; e++) {
            const T* lo = e == 0 ? b1 : bc;
            const T* hi = e == 0 ? bc : bp1;
            T W[NW][N], s[NW], am[N], ap[N];
            typename RP::Lin L;
            solve_pair<RP, O>(rp, lo, hi, W, s, am, ap, L);
            // the low edge's A+dQ and the high edge's A-dQ enter the cell
            T X[N];
#pragma unroll
            for (int m = 0; m < N; m++) X[m] = e == 0 ? ap[m] : am[m];
            if (t2) {
                T c[N];
                if (e == 0) correction4<RP, O>(rp, b2, b1, bc, bp1, dto, S.limiter, c);
                else correction4<RP, O>(rp, b1, bc, bp1, bp2, dto, S.limiter, c);
#pragma unroll
                for (int m = 0; m < N; m++) X[m] += e == 0 ? -c[m] : c[m];
            }
            T bm[N], bpq[N];
            rp.template transverse<O>(L, X, bm, bpq);
#pragma unroll
            for (int m = 0; m < N; m++) F[m] -= T(0.5) * dto * (side == 1 ? bm[m] : bpq[m]);
        }
    }
}

}  // namespace mc
