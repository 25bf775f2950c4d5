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

// ---------------------------------------------------- bounds-checked debug build
// Compiled with -DLBCG_CHECK_BOUNDS, every population, link-word and psi-ring index of the
// step kernels is checked before the access: an index outside its array sets the context's
// status word to kStatusBounds (lbcg_synchronize and the read-backs then report
// LBCG_ERR_BOUNDS) and the access is skipped (a load reads 0), so a faulty index is reported
// instead of faulting the GPU.  Without the flag the checks compile to nothing.
constexpr int kStatusTimeout = 1, kStatusBounds = 2;

__device__ __forceinline__ bool in_bounds(const KParams& P, long long i, long long n)
{
#ifdef LBCG_CHECK_BOUNDS
    if (i < 0 || i >= n) {
        if (P.status) atomicExch(P.status, kStatusBounds);
        return false;
    }
#endif
    (void)P;
    (void)i;
    (void)n;
    return true;
}

// elements of one state buffer (2Q planes of np values)
__device__ __forceinline__ long long state_elems(const KParams& P) { return (P.lattice ? 38LL : 18LL) * (long long)P.np; }
// sites of the box (link words)
__device__ __forceinline__ long long box_sites(const KParams& P) { return (long long)P.nx * P.ny * P.nz; }

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
    // the two stored values of one direction (what store writes)
    __device__ static __forceinline__ void encode(T r, T g, const Phys<T>& ph, int c, S& fr, S& fb)
    {
        fr = (S)r;
        fb = (S)((g + ph.wr0[c]) - r);
    }
    template <typename IDX>
    __device__ static __forceinline__ void store(S* __restrict__ b, IDX ir, IDX ig, const Phys<T>& ph, int c, T r,
                                                 T g)
    {
        encode(r, g, ph, c, b[ir], b[ig]);
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
    __device__ static __forceinline__ void encode(T r, T g, const Phys<T>&, int, S& fr, S& fg)
    {
        fr = r;
        fg = g;
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
    __device__ static __forceinline__ void decode(S fr, S fg, const Phys<T>& ph, int c, T& r, T& g)
    {
        const float wi = ph.w[c];
        r = __half2float(fr) * wi + 0.5f * ph.wr0[c];
        g = __half2float(fg) * (wi * ph.inv_scale_g);
    }
    __device__ static __forceinline__ void encode(T r, T g, const Phys<T>& ph, int c, S& fr, S& fg)
    {
        const float iw = ph.inv_w[c];
        fr = __float2half_rn((r - 0.5f * ph.wr0[c]) * iw);
        fg = __float2half_rn(g * (iw * ph.scale_g));
    }
    template <typename IDX>
    __device__ static __forceinline__ void store(S* __restrict__ b, IDX ir, IDX ig, const Phys<T>& ph, int c, T r,
                                                 T g)
    {
        encode(r, g, ph, c, b[ir], b[ig]);
    }
};

// population access through the bounds checks (ir: red-plane element, ig: second-plane element)
template <int PREC, typename IDX>
__device__ __forceinline__ void load_pop(const KParams& P, const typename Store<PREC>::S* __restrict__ a, IDX ir,
                                         IDX ig, const Phys<typename Store<PREC>::T>& ph, int c,
                                         typename Store<PREC>::T& r, typename Store<PREC>::T& g)
{
#ifdef LBCG_CHECK_BOUNDS
    const long long n = state_elems(P);
    if (!in_bounds(P, (long long)ir, n) || !in_bounds(P, (long long)ig, n)) {
        r = g = 0;
        return;
    }
#endif
    Store<PREC>::load(a, ir, ig, ph, c, r, g);
}

template <int PREC, typename IDX>
__device__ __forceinline__ void store_pop(const KParams& P, typename Store<PREC>::S* __restrict__ b, IDX ir, IDX ig,
                                          const Phys<typename Store<PREC>::T>& ph, int c, typename Store<PREC>::T r,
                                          typename Store<PREC>::T g)
{
#ifdef LBCG_CHECK_BOUNDS
    const long long n = state_elems(P);
    if (!in_bounds(P, (long long)ir, n) || !in_bounds(P, (long long)ig, n)) return;
#endif
    Store<PREC>::store(b, ir, ig, ph, c, r, g);
}

// link word of site s (0 without a link table)
template <typename IDX>
__device__ __forceinline__ uint32_t load_link(const KParams& P, const uint32_t* __restrict__ link, IDX s)
{
    if (!link || !in_bounds(P, (long long)s, box_sites(P))) return 0u;
    return __ldg(link + s);
}

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

// psi of a port ghost site from its own populations: the rest population, then opposite
// pairs (one summation order for every kernel and for the refill's ghost-psi table)
template <int LAT, typename T, typename LD>
__device__ __forceinline__ T ghost_psi_from(const Phys<T>& ph, LD&& ld)
{
    using L = Lat<LAT>;
    T rr, sg;
    ld(0, rr, sg);
#pragma unroll
    for (int k = 0; k < L::NP; ++k) {
        const int p = L::rep(k);
        T rp, gp, rq, gq;
        ld(p, rp, gp);
        ld(L::opp(p), rq, gq);
        rr += rp + rq;
        sg += gp + gq;
    }
    const T rho = ph.rho0 + sg;
    return (rr - (rho - rr)) / rho;
}

template <int LAT, int PREC, typename IDX>
__device__ __forceinline__ typename Store<PREC>::T ghost_psi(const KParams& P,
                                                             const typename Store<PREC>::S* __restrict__ A, IDX s)
{
    using L = Lat<LAT>;
    using T = typename Store<PREC>::T;
    const IDX np = (IDX)P.np;
    return ghost_psi_from<LAT, T>(phys<T>(P), [&](int i, T& r, T& g) {
        const IDX ir = (IDX)i * np + s;
        load_pop<PREC, IDX>(P, A, ir, ir + (IDX)L::Q * np, phys<T>(P), L::cls(i), r, g);
    });
}

// ------------------------------------------------------------ port ghost refill
// Ghost g of port m, inward neighbour x' (a fluid site):
//   velocity:      f^k = f^{k,eq}(chi^k rho', u_port) + chi^k (f(x') - f^eq(x'))
//   pressure:      f^k = f^{k,eq}(rho_port rho'^k / rho', u') + f^k(x') - f^{k,eq}(x')
//   zero-gradient: f^k = f^k(x')
// One thread per ghost, in the storage format's compute type, on the register form
// (r_i = f^R_i, g_i = f_i - w_i rho0): every quantity formed is a small deviation, so
// FP32 keeps the precision of the stored populations.  With phi^k_i = w_i + dphi^k_i and
// P_i(u) = 3 c.u + 4.5 (c.u)^2 - 1.5 u^2:
//   f^eq_i - w_i rho0 = w_i (rho - rho0) + rho_R dphi^R_i + rho_B dphi^B_i + w_i rho P_i(u),
//   f^{R,eq}_i(rho_R, u) = rho_R (phi^R_i + w_i P_i(u)),
// and the pressure rule reduces to f^k_i(x') + (rho_port / rho' - 1) f^{k,eq}_i(x').
template <int LAT, int PREC>
__device__ __forceinline__ void fill_one(const KParams& P, typename Store<PREC>::S* __restrict__ a,
                                         const int* __restrict__ tab, const double* __restrict__ gu, int ng, int t,
                                         typename Store<PREC>::T* __restrict__ gpsi = nullptr)
{
    using L = Lat<LAT>;
    using SP = Store<PREC>;
    using T = typename SP::T;
    constexpr int Q = L::Q;
    const Phys<T>& ph = phys<T>(P);
    const size_t np = P.np;
    const size_t g = (size_t)tab[t];
    const size_t xp = (size_t)tab[ng + t];
    const int kind = tab[3 * ng + t];
    T r[Q], d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) SP::load(a, i * np + xp, (Q + i) * np + xp, ph, L::cls(i), r[i], d[i]);
    // Every direction is stored through put, in index order.  With a ghost-psi table the stored
    // values are decoded as a later load would decode them and summed in the order of
    // ghost_psi_from (rest, then each opposite pair), so the table holds the bits ghost_psi would
    // compute.  D3Q19, whose opposite directions are the consecutive pairs (1, 2) .. (17, 18),
    // sums as it stores (the fused refill runs inside the register budget of the march); D2Q9,
    // refilled by separate kernels only, keeps the decoded values and sums them at the end.
    static_assert(LAT != 1 || (L::rep(0) == 1 && L::opp(1) == 2 && L::rep(8) == 17 && L::opp(17) == 18),
                  "D3Q19 opposite pairs must be consecutive");
    T sr = 0, sd = 0, hr = 0, hd = 0;
    T kr[LAT == 0 ? Q : 1], kd[LAT == 0 ? Q : 1];
    auto put = [&](int i, int c, T vr, T vd) {
        typename SP::S fr, fd;
        SP::encode(vr, vd, ph, c, fr, fd);
        a[i * np + g] = fr;
        a[(Q + i) * np + g] = fd;
        if (!gpsi) return;
        T er, ed;
        SP::decode(fr, fd, ph, c, er, ed);
        if (LAT == 0) {
            kr[LAT == 0 ? i : 0] = er;
            kd[LAT == 0 ? i : 0] = ed;
        } else if (i == 0) {
            sr = er;
            sd = ed;
        } else if (i & 1) {
            hr = er;
            hd = ed;
        } else {
            sr += hr + er;
            sd += hd + ed;
        }
    };
    auto finish = [&]() {
        if (!gpsi) return;
        if (LAT == 0) {
            gpsi[t] = ghost_psi_from<LAT, T>(ph, [&](int i, T& r, T& d) {
                r = kr[LAT == 0 ? i : 0];
                d = kd[LAT == 0 ? i : 0];
            });
            return;
        }
        const T rho = ph.rho0 + sd;
        gpsi[t] = (sr - (rho - sr)) / rho;
    };
    if (kind == LBCG_PORT_ZERO_GRADIENT) {
#pragma unroll
        for (int i = 0; i < Q; ++i) put(i, L::cls(i), r[i], d[i]);
        finish();
        return;
    }
    T rr = 0, dr = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        rr += r[i];
        dr += d[i];
        if (L::cx(i)) jx += L::cx(i) > 0 ? d[i] : -d[i];
        if (L::cy(i)) jy += L::cy(i) > 0 ? d[i] : -d[i];
        if (L::cz(i)) jz += L::cz(i) > 0 ? d[i] : -d[i];
    }
    const T rho = ph.rho0 + dr;
    const T rb = rho - rr;
    const T inv_rho = T(1) / rho;
    const T ux = jx * inv_rho, uy = jy * inv_rho, uz = jz * inv_rho;
    const T usq = ux * ux + uy * uy + uz * uz;
    if (kind == LBCG_PORT_VELOCITY) {
        const T vx = (T)gu[t], vy = (T)gu[ng + t], vz = (T)gu[2 * ng + t];
        const T psi = (T)gu[4 * ng + t];
        const T xr = (T(1) + psi) * T(0.5), xb = (T(1) - psi) * T(0.5);
        const T vsq = vx * vx + vy * vy + vz * vz;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int c = L::cls(i);
            const T wi = (T)L::w(i);
            const T cu = (T)L::cx(i) * ux + (T)L::cy(i) * uy + (T)L::cz(i) * uz;
            const T cv = (T)L::cx(i) * vx + (T)L::cy(i) * vy + (T)L::cz(i) * vz;
            const T pu = T(3) * cu + T(4.5) * cu * cu - T(1.5) * usq;
            const T pv = T(3) * cv + T(4.5) * cv * cv - T(1.5) * vsq;
            const T neq = d[i] - (wi * dr + rr * ph.dphiR[c] + rb * ph.dphiB[c] + wi * rho * pu);
            const T gr = xr * rho * (ph.phiR[c] + wi * pv) + xr * neq;
            const T gd = wi * dr + xr * rho * ph.dphiR[c] + xb * rho * ph.dphiB[c] + wi * rho * pv + neq;
            put(i, c, gr, gd);
        }
    } else {
        const T fac = (T)gu[3 * ng + t] * inv_rho - T(1);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int c = L::cls(i);
            const T wi = (T)L::w(i);
            const T cu = (T)L::cx(i) * ux + (T)L::cy(i) * uy + (T)L::cz(i) * uz;
            const T pu = wi * (T(3) * cu + T(4.5) * cu * cu - T(1.5) * usq);
            const T er = rr * (ph.phiR[c] + pu), eb = rb * (ph.phiB[c] + pu);
            put(i, c, r[i] + fac * er, d[i] + fac * (er + eb));
        }
    }
    finish();  // the ghost's psi for the next step's colour gradient
}

}  // namespace lbcg
