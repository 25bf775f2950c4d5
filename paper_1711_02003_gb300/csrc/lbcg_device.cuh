// lbcg_device.cuh -- device-side lattice constants, population storage formats and
// the per-site regularized colour-gradient collision (arXiv:1711.02003, Sec. II).
//
// Everything here is written for sm_103a and is independent of the FP64 oracle.
#pragma once

#include <cuda_fp16.h>
#include <cstdint>

#include "lbcg_internal.h"

namespace lbcg {

// ------------------------------------------------------------------------- lattices
// Directions are 0-based (0 = rest) in the order documented in include/lbcg.h.
// Speed class: 0 rest, 1 axis/face (|c|^2 = 1), 2 diagonal/edge (|c|^2 = 2).

template <int LAT>
struct Lat;

template <>
struct Lat<0> {  // D2Q9
    static constexpr int D = 2, Q = 9;
    __host__ __device__ static constexpr int cx(int i)
    {
        return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0);
    }
    __host__ __device__ static constexpr int cy(int i)
    {
        return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0);
    }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr int cls(int i) { return i == 0 ? 0 : (i < 5 ? 1 : 2); }
    __host__ __device__ static constexpr int opp(int i)
    {
        return i == 0 ? 0 : (i < 5 ? (i + 1) % 4 + 1 : (i + 1) % 4 + 5);
    }
    // lattice weights w_i and the perturbation constants B_i of Eq. 9 per speed class
    __host__ __device__ static constexpr double w(int i)
    {
        return cls(i) == 0 ? 4.0 / 9.0 : (cls(i) == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
    __host__ __device__ static constexpr double Bc(int i)
    {
        return cls(i) == 0 ? -4.0 / 27.0 : (cls(i) == 1 ? 2.0 / 27.0 : 5.0 / 108.0);
    }
    // opposite-direction pairs (p, opp(p)): p = rep(k)
    static constexpr int NP = 4;
    __host__ __device__ static constexpr int rep(int k) { return k == 0 ? 1 : (k == 1 ? 2 : (k == 2 ? 5 : 6)); }
};

template <>
struct Lat<1> {  // D3Q19
    static constexpr int D = 3, Q = 19;
    // faces 1..6: +x -x +y -y +z -z; edges 7..18 in pairs (v, -v)
    __host__ __device__ static constexpr int cx(int i)
    {
        return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
             : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
    }
    __host__ __device__ static constexpr int cy(int i)
    {
        return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
             : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
    }
    __host__ __device__ static constexpr int cz(int i)
    {
        return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
             : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
    }
    __host__ __device__ static constexpr int cls(int i) { return i == 0 ? 0 : (i < 7 ? 1 : 2); }
    __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
    __host__ __device__ static constexpr double w(int i)
    {
        return cls(i) == 0 ? 1.0 / 3.0 : (cls(i) == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
    __host__ __device__ static constexpr double Bc(int i)
    {
        return cls(i) == 0 ? -1.0 / 3.0 : (cls(i) == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
    static constexpr int NP = 9;
    __host__ __device__ static constexpr int rep(int k) { return 2 * k + 1; }
};

// ---------------------------------------------------------------- storage formats
// In registers every format becomes (r_i, g_i): r_i = f^R_i (red population) and
// g_i = f^R_i + f^B_i - w_i rho0 (total deviation).  The collision works on these.
// load/store take the direction's speed class c (for w_i rho0 and 1/w_i).

template <int PREC>
struct Store;

template <typename S_, typename T_>
struct StorePlain {
    using S = S_;
    using T = T_;
    // ir: element index of direction i's red plane at the site; ig: of its second plane
    template <typename IDX>
    __device__ static __forceinline__ void load(const S* __restrict__ a, IDX ir, IDX ig, const Phys<T>& ph, int c,
                                                T& r, T& g)
    {
        const T fr = (T)a[ir];
        const T fb = (T)a[ig];
        r = fr;
        g = (fr + fb) - ph.wr0[c];
    }
    template <typename IDX>
    __device__ static __forceinline__ void store(S* __restrict__ b, IDX ir, IDX ig, const Phys<T>& ph, int c, T r,
                                                 T g)
    {
        b[ir] = (S)r;
        b[ig] = (S)((g + ph.wr0[c]) - r);
    }
    // register form of the two stored values of one direction (as load)
    __device__ static __forceinline__ void decode(S fr_, S fb_, const Phys<T>& ph, int c, T& r, T& g)
    {
        const T fr = (T)fr_, fb = (T)fb_;
        r = fr;
        g = (fr + fb) - ph.wr0[c];
    }
};

template <>
struct Store<LBCG_FP64> : StorePlain<double, double> {};
template <>
struct Store<LBCG_FP32> : StorePlain<float, float> {};

template <>
struct Store<LBCG_FP32_DEV> {
    using S = float;
    using T = float;
    template <typename IDX>
    __device__ static __forceinline__ void load(const S* __restrict__ a, IDX ir, IDX ig, const Phys<T>&, int, T& r,
                                                T& g)
    {
        r = a[ir];
        g = a[ig];
    }
    template <typename IDX>
    __device__ static __forceinline__ void store(S* __restrict__ b, IDX ir, IDX ig, const Phys<T>&, int, T r, T g)
    {
        b[ir] = r;
        b[ig] = g;
    }
    __device__ static __forceinline__ void decode(S fr, S fg, const Phys<T>&, int, T& r, T& g)
    {
        r = fr;
        g = fg;
    }
};

// binary16: red as (f^R_i - w_i rho0/2) / w_i and total deviation g_i / w_i * scale_g,
// so every direction spans the same range; decoded to FP32.
template <>
struct Store<LBCG_FP16_SCALED> {
    using S = __half;
    using T = float;
    __device__ static __forceinline__ float wcls(int c, const Phys<T>& ph) { return ph.wr0[c] / ph.rho0; }
    template <typename IDX>
    __device__ static __forceinline__ void load(const S* __restrict__ a, IDX ir, IDX ig, const Phys<T>& ph, int c,
                                                T& r, T& g)
    {
        const float wi = ph.w[c];
        r = __half2float(a[ir]) * wi + 0.5f * ph.wr0[c];
        g = __half2float(a[ig]) * (wi * ph.inv_scale_g);
    }
    template <typename IDX>
    __device__ static __forceinline__ void store(S* __restrict__ b, IDX ir, IDX ig, const Phys<T>& ph, int c, T r,
                                                 T g)
    {
        const float iw = ph.inv_w[c];
        b[ir] = __float2half_rn((r - 0.5f * ph.wr0[c]) * iw);
        b[ig] = __float2half_rn(g * (iw * ph.scale_g));
    }
};

// ------------------------------------------------------------------ the collision
// One fluid site.  In: r[i], g[i] post-streaming (Eq. 1), the colour gradient F.
// Out: r[i] = post-collision red population, g[i] = post-collision total deviation.
// Steps (Eq. 4 read as a sequence): moments (Eqs. 2-3), mixture relaxation time,
// equilibrium (Eqs. 6-7), regularized relaxation (Eq. 11) or BGK (Eq. 5),
// perturbation (Eq. 9), recolouring (Eq. 10).
//
// Evaluation by opposite-direction pairs (p, q = opp(p), c_q = -c_p): the
// equilibrium, the Hermite term of Eq. 11 and the perturbation are sums of a part
// even in c (shared by p and q) and a part odd in c (equal and opposite), so each
// pair is computed once: g_p = S + A, g_q = S - A; the recolouring split likewise
// r_p = X + Y, r_q = X - Y.  The second moment Pi of the non-equilibrium only sees
// the even parts.  The same quantities as a direction-by-direction evaluation, in
// fewer operations.
template <int LAT, typename T>
__device__ __forceinline__ void collide_site(const KParams& P, const Phys<T>& ph, T (&r)[Lat<LAT>::Q],
                                             T (&g)[Lat<LAT>::Q], const T F[3])
{
    using L = Lat<LAT>;
    constexpr int NP = L::NP;
    const T rho0 = ph.rho0;

    // moments (Eqs. 2-3)
    T rhoR = r[0], sg = g[0], jx = 0, jy = 0, jz = 0;
    T ge[NP], go[NP];  // even and odd halves of each pair
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int p = L::rep(k), q = L::opp(p);
        rhoR += r[p] + r[q];
        ge[k] = g[p] + g[q];
        go[k] = g[p] - g[q];
        sg += ge[k];
        if (L::cx(p)) jx += L::cx(p) > 0 ? go[k] : -go[k];
        if (L::cy(p)) jy += L::cy(p) > 0 ? go[k] : -go[k];
        if (L::D == 3 && L::cz(p)) jz += L::cz(p) > 0 ? go[k] : -go[k];
    }
    const T rho = rho0 + sg;
    const T rhoB = rho - rhoR;
    const T inv_rho = T(1) / rho;
    const T ux = jx * inv_rho, uy = jy * inv_rho, uz = jz * inv_rho;
    const T psi = (rhoR - rhoB) * inv_rho;

    // mixture viscosity 1/nu = (1+psi)/(2 nu_R) + (1-psi)/(2 nu_B); tau = 3 nu + 1/2
    const T inv_nu = (T(1) + psi) * ph.half_inv_nu_r + (T(1) - psi) * ph.half_inv_nu_b;
    const T tau = T(3) / inv_nu + T(0.5);
    const T om1 = T(1) - T(1) / tau;

    // equilibrium (Eqs. 6-7) as deviation from w_i rho0: even part eS, odd part eA
    const T usq = ux * ux + uy * uy + uz * uz;
    const T base = sg - T(1.5) * rho * usq;              // drho - 1.5 rho u^2
    const T dphi0 = rhoR * ph.dphiR[0] + rhoB * ph.dphiB[0];
    const T dphi1 = rhoR * ph.dphiR[1] + rhoB * ph.dphiB[1];
    const T dphi2 = rhoR * ph.dphiR[2] + rhoB * ph.dphiB[2];
    const T eq0 = (T)L::w(0) * base + dphi0;
    T eS[NP], eA[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int p = L::rep(k);
        const T cu = (T)L::cx(p) * ux + (T)L::cy(p) * uy + (T)L::cz(p) * uz;
        const T wi = (T)L::w(p);
        eS[k] = wi * (base + T(4.5) * rho * cu * cu) + (L::cls(p) == 1 ? dphi1 : dphi2);
        eA[k] = (T(3) * wi) * rho * cu;
    }

    T gS[NP], gA[NP], g0;
    if (P.collision == LBCG_BGK) {
        g0 = eq0 + om1 * (g[0] - eq0);
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            gS[k] = eS[k] + om1 * (T(0.5) * ge[k] - eS[k]);
            gA[k] = eA[k] + om1 * (T(0.5) * go[k] - eA[k]);
        }
    } else {
        // Pi^neq = sum_i (g_i - geq_i) c_i c_i: only even parts contribute
        T pxx = 0, pyy = 0, pzz = 0, pxy = 0, pxz = 0, pyz = 0;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const int p = L::rep(k);
            const T ne = ge[k] - T(2) * eS[k];
            const int ax = L::cx(p), ay = L::cy(p), az = L::cz(p);
            if (ax) pxx += ne;
            if (ay) pyy += ne;
            if (az) pzz += ne;
            if (ax && ay) pxy += (ax * ay > 0) ? ne : -ne;
            if (ax && az) pxz += (ax * az > 0) ? ne : -ne;
            if (ay && az) pyz += (ay * az > 0) ? ne : -ne;
        }
        const T tr3 = (pxx + pyy + pzz) * (T(1) / T(3));
        g0 = eq0 + om1 * (T(4.5) * (T)L::w(0)) * (-tr3);
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const int p = L::rep(k);
            const int ax = L::cx(p), ay = L::cy(p), az = L::cz(p);
            T qp = -tr3;
            if (ax) qp += pxx;
            if (ay) qp += pyy;
            if (az) qp += pzz;
            if (ax && ay) qp += T(2 * ax * ay) * pxy;
            if (ax && az) qp += T(2 * ax * az) * pxz;
            if (ay && az) qp += T(2 * ay * az) * pyz;
            gS[k] = eS[k] + om1 * (T(4.5) * (T)L::w(p)) * qp;
            gA[k] = eA[k];
        }
    }

    // perturbation (Eq. 9): even in c
    const T fn2 = F[0] * F[0] + F[1] * F[1] + F[2] * F[2];
    const bool has_f = fn2 > T(1e-20);
    const T fn = has_f ? sqrt(fn2) : T(0);
    const T inv_fn = has_f ? T(1) / fn : T(0);
    const T inv_fn2 = inv_fn * inv_fn;
    const T half_a_fn = T(0.5) * ph.A * fn;
    T fcs[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int p = L::rep(k);
        fcs[k] = (T)L::cx(p) * F[0] + (T)L::cy(p) * F[1] + (T)L::cz(p) * F[2];
        if (has_f) gS[k] += half_a_fn * ((T)L::w(p) * fcs[k] * fcs[k] * inv_fn2 - (T)L::Bc(p));
    }
    if (has_f) g0 -= half_a_fn * (T)L::Bc(0);

    // recolouring (Eq. 10).  It keeps rho_R of the site exactly; the rest direction
    // (cos phi_0 = 0) takes rho_R minus the other directions, so the FP32 rounding of
    // the sum cannot repeat step after step at a static interface and drift.
    const T seg = ph.beta * rhoR * rhoB * inv_rho * inv_rho;
    const T fracR = rhoR * inv_rho;
    const T inv_sqrt2 = T(0.70710678118654752440);
    const T e1 = rhoR * ph.phiR[1] + rhoB * ph.phiB[1];
    const T e2 = rhoR * ph.phiR[2] + rhoB * ph.phiB[2];
    T rsum = 0;
    g[0] = g0;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int p = L::rep(k), q = L::opp(p);
        const int c = L::cls(p);
        const T cosphi = c == 1 ? fcs[k] * inv_fn : fcs[k] * inv_fn * inv_sqrt2;
        const T X = fracR * (gS[k] + ph.wr0[c]);
        const T Y = fracR * gA[k] + seg * cosphi * (c == 1 ? e1 : e2);
        g[p] = gS[k] + gA[k];
        g[q] = gS[k] - gA[k];
        r[p] = X + Y;
        r[q] = X - Y;
        rsum += r[p] + r[q];
    }
    r[0] = rhoR - rsum;
}


// ------------------------------------------------------- the collision from moments
// The regularized collision (Eq. 11) rebuilds every post-collision population from the
// site's moments: rho_R, rho, the momentum, the second moment Pi of the streamed
// populations, and the colour gradient F.  None of the individual streamed
// populations is needed once these are summed, so a kernel can accumulate them while
// the pulled populations arrive and keep 11 numbers per waiting site instead of 2Q.
// The arithmetic is that of collide_site's regularized branch; only the order of the
// sums differs (Pi^neq = Pi - Pi^eq instead of sum_i (f_i - feq_i) c_i c_i).
template <typename T>
struct SiteMom {
    T rr, sg;                        // rho_R; rho - rho0 (sum of the total deviations g_i)
    T jx, jy, jz;                    // momentum (sum_i g_i c_i)
    T pxx, pyy, pzz, pxy, pxz, pyz;  // sum_i g_i c_ia c_ib
};

template <typename T>
__device__ __forceinline__ void mom_zero(SiteMom<T>& m)
{
    m.rr = m.sg = m.jx = m.jy = m.jz = T(0);
    m.pxx = m.pyy = m.pzz = m.pxy = m.pxz = m.pyz = T(0);
}

// add the opposite pair (p = rep(k), opp(p)); FULL = false sums only rho_R and rho
template <int LAT, bool FULL, typename T>
__device__ __forceinline__ void mom_add_pair(SiteMom<T>& m, int k, T rp, T gp, T rq, T gq)
{
    using L = Lat<LAT>;
    const int p = L::rep(k);
    m.rr += rp + rq;
    const T ge = gp + gq;
    m.sg += ge;
    if (!FULL) return;
    const T go = gp - gq;
    const int ax = L::cx(p), ay = L::cy(p), az = L::cz(p);
    if (ax) m.jx += ax > 0 ? go : -go;
    if (ay) m.jy += ay > 0 ? go : -go;
    if (az) m.jz += az > 0 ? go : -go;
    if (ax) m.pxx += ge;
    if (ay) m.pyy += ge;
    if (az) m.pzz += ge;
    if (ax && ay) m.pxy += (ax * ay > 0) ? ge : -ge;
    if (ax && az) m.pxz += (ax * az > 0) ? ge : -ge;
    if (ay && az) m.pyz += (ay * az > 0) ? ge : -ge;
}

// Regularized collision, perturbation and recolouring of one site from its moments;
// out(i, r_i, g_i) receives every post-collision population (the rest direction last).
template <int LAT, typename T, typename Out>
__device__ __forceinline__ void collide_moments(const Phys<T>& ph, const SiteMom<T>& m, const T F[3], Out&& out)
{
    using L = Lat<LAT>;
    constexpr int NP = L::NP;
    const T rhoR = m.rr, sg = m.sg;
    const T rho = ph.rho0 + sg;
    const T rhoB = rho - rhoR;
    const T inv_rho = T(1) / rho;
    const T ux = m.jx * inv_rho, uy = m.jy * inv_rho, uz = L::D == 3 ? m.jz * inv_rho : T(0);
    const T psi = (rhoR - rhoB) * inv_rho;

    const T inv_nu = (T(1) + psi) * ph.half_inv_nu_r + (T(1) - psi) * ph.half_inv_nu_b;
    const T tau = T(3) / inv_nu + T(0.5);
    const T om1 = T(1) - T(1) / tau;

    // equilibrium (Eqs. 6-7) as deviation from w_i rho0, even part per pair; its second
    // moment is taken off Pi to leave Pi^neq
    const T usq = ux * ux + uy * uy + uz * uz;
    const T base = sg - T(1.5) * rho * usq;
    const T dphi0 = rhoR * ph.dphiR[0] + rhoB * ph.dphiB[0];
    const T dphi1 = rhoR * ph.dphiR[1] + rhoB * ph.dphiB[1];
    const T dphi2 = rhoR * ph.dphiR[2] + rhoB * ph.dphiB[2];
    const T eq0 = (T)L::w(0) * base + dphi0;
    T qxx = m.pxx, qyy = m.pyy, qzz = m.pzz, qxy = m.pxy, qxz = m.pxz, qyz = m.pyz;
    T eS[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int p = L::rep(k);
        const int ax = L::cx(p), ay = L::cy(p), az = L::cz(p);
        const T cu = (T)ax * ux + (T)ay * uy + (T)az * uz;
        eS[k] = (T)L::w(p) * (base + T(4.5) * rho * cu * cu) + (L::cls(p) == 1 ? dphi1 : dphi2);
        const T e = T(2) * eS[k];
        if (ax) qxx -= e;
        if (ay) qyy -= e;
        if (az) qzz -= e;
        if (ax && ay) qxy -= (ax * ay > 0) ? e : -e;
        if (ax && az) qxz -= (ax * az > 0) ? e : -e;
        if (ay && az) qyz -= (ay * az > 0) ? e : -e;
    }
    const T tr3 = (qxx + qyy + qzz) * (T(1) / T(3));
    T g0 = eq0 + om1 * (T(4.5) * (T)L::w(0)) * (-tr3);

    // perturbation (Eq. 9)
    const T fn2 = F[0] * F[0] + F[1] * F[1] + F[2] * F[2];
    const bool has_f = fn2 > T(1e-20);
    const T fn = has_f ? sqrt(fn2) : T(0);
    const T inv_fn = has_f ? T(1) / fn : T(0);
    const T inv_fn2 = inv_fn * inv_fn;
    const T half_a_fn = T(0.5) * ph.A * fn;
    if (has_f) g0 -= half_a_fn * (T)L::Bc(0);

    // recolouring (Eq. 10); the rest direction takes rho_R minus the others
    const T seg = ph.beta * rhoR * rhoB * inv_rho * inv_rho;
    const T fracR = rhoR * inv_rho;
    const T inv_sqrt2 = T(0.70710678118654752440);
    const T ew1 = rhoR * ph.phiR[1] + rhoB * ph.phiB[1];
    const T ew2 = rhoR * ph.phiR[2] + rhoB * ph.phiB[2];
    T rsum = 0;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int p = L::rep(k), q = L::opp(p);
        const int ax = L::cx(p), ay = L::cy(p), az = L::cz(p);
        const int c = L::cls(p);
        T qp = -tr3;
        if (ax) qp += qxx;
        if (ay) qp += qyy;
        if (az) qp += qzz;
        if (ax && ay) qp += T(2 * ax * ay) * qxy;
        if (ax && az) qp += T(2 * ax * az) * qxz;
        if (ay && az) qp += T(2 * ay * az) * qyz;
        const T cu = (T)ax * ux + (T)ay * uy + (T)az * uz;
        T gS = eS[k] + om1 * (T(4.5) * (T)L::w(p)) * qp;
        const T gA = (T(3) * (T)L::w(p)) * rho * cu;
        const T fcs = (T)ax * F[0] + (T)ay * F[1] + (T)az * F[2];
        if (has_f) gS += half_a_fn * ((T)L::w(p) * fcs * fcs * inv_fn2 - (T)L::Bc(p));
        const T cosphi = c == 1 ? fcs * inv_fn : fcs * inv_fn * inv_sqrt2;
        const T X = fracR * (gS + ph.wr0[c]);
        const T Y = fracR * gA + seg * cosphi * (c == 1 ? ew1 : ew2);
        const T rp = X + Y, rq = X - Y;
        out(p, rp, gS + gA);
        out(q, rq, gS - gA);
        rsum += rp + rq;
    }
    out(0, rhoR - rsum, g0);
}

}  // namespace lbcg
