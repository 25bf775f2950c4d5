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
    __device__ static __forceinline__ void load(const S* __restrict__ a, size_t np, int Q, int i, size_t s,
                                                const Phys<T>& ph, int c, T& r, T& g)
    {
        const T fr = (T)a[(size_t)i * np + s];
        const T fb = (T)a[(size_t)(Q + i) * np + s];
        r = fr;
        g = (fr + fb) - ph.wr0[c];
    }
    __device__ static __forceinline__ void store(S* __restrict__ b, size_t np, int Q, int i, size_t s,
                                                 const Phys<T>& ph, int c, T r, T g)
    {
        b[(size_t)i * np + s] = (S)r;
        b[(size_t)(Q + i) * np + s] = (S)((g + ph.wr0[c]) - r);
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
    __device__ static __forceinline__ void load(const S* __restrict__ a, size_t np, int Q, int i, size_t s,
                                                const Phys<T>&, int, T& r, T& g)
    {
        r = a[(size_t)i * np + s];
        g = a[(size_t)(Q + i) * np + s];
    }
    __device__ static __forceinline__ void store(S* __restrict__ b, size_t np, int Q, int i, size_t s,
                                                 const Phys<T>&, int, T r, T g)
    {
        b[(size_t)i * np + s] = r;
        b[(size_t)(Q + i) * np + s] = g;
    }
};

// binary16: red as (f^R_i - w_i rho0/2) / w_i and total deviation g_i / w_i * scale_g,
// so every direction spans the same range; decoded to FP32.
template <>
struct Store<LBCG_FP16_SCALED> {
    using S = __half;
    using T = float;
    __device__ static __forceinline__ float wcls(int Q, int c)
    {
        return Q == 9 ? (c == 0 ? 4.0f / 9.0f : (c == 1 ? 1.0f / 9.0f : 1.0f / 36.0f))
                      : (c == 0 ? 1.0f / 3.0f : (c == 1 ? 1.0f / 18.0f : 1.0f / 36.0f));
    }
    __device__ static __forceinline__ float iwcls(int Q, int c)
    {
        return Q == 9 ? (c == 0 ? 2.25f : (c == 1 ? 9.0f : 36.0f)) : (c == 0 ? 3.0f : (c == 1 ? 18.0f : 36.0f));
    }
    __device__ static __forceinline__ void load(const S* __restrict__ a, size_t np, int Q, int i, size_t s,
                                                const Phys<T>& ph, int c, T& r, T& g)
    {
        const float wi = wcls(Q, c);
        r = __half2float(a[(size_t)i * np + s]) * wi + 0.5f * ph.wr0[c];
        g = __half2float(a[(size_t)(Q + i) * np + s]) * (wi * ph.inv_scale_g);
    }
    __device__ static __forceinline__ void store(S* __restrict__ b, size_t np, int Q, int i, size_t s,
                                                 const Phys<T>& ph, int c, T r, T g)
    {
        const float iw = iwcls(Q, c);
        b[(size_t)i * np + s] = __float2half_rn((r - 0.5f * ph.wr0[c]) * iw);
        b[(size_t)(Q + i) * np + s] = __float2half_rn(g * (iw * ph.scale_g));
    }
};

// ------------------------------------------------------------------ the collision
// One fluid site.  In: r[i], g[i] post-streaming (Eq. 1), the colour gradient F.
// Out: r[i] = post-collision red population, g[i] = post-collision total deviation.
// Steps (Eq. 4 read as a sequence): moments (Eqs. 2-3), mixture relaxation time,
// equilibrium (Eqs. 6-7), regularized relaxation (Eq. 11) or BGK (Eq. 5),
// perturbation (Eq. 9), recolouring (Eq. 10).
template <int LAT, typename T>
__device__ __forceinline__ void collide_site(const KParams& P, const Phys<T>& ph, T (&r)[Lat<LAT>::Q],
                                             T (&g)[Lat<LAT>::Q], const T F[3])
{
    using L = Lat<LAT>;
    constexpr int Q = L::Q;
    const T rho0 = ph.rho0;

    T rhoR = 0, sg = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        rhoR += r[i];
        sg += g[i];
        if (L::cx(i)) jx += L::cx(i) > 0 ? g[i] : -g[i];
        if (L::cy(i)) jy += L::cy(i) > 0 ? g[i] : -g[i];
        if (L::D == 3 && L::cz(i)) jz += L::cz(i) > 0 ? g[i] : -g[i];
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

    const T usq = ux * ux + uy * uy + uz * uz;
    const T drho = sg;  // rho - rho0
    T geq[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T cu = (T)L::cx(i) * ux + (T)L::cy(i) * uy + (T)L::cz(i) * uz;
        const T wi = (T)L::w(i);
        const int c = L::cls(i);
        const T dphi = rhoR * ph.dphiR[c] + rhoB * ph.dphiB[c];
        geq[i] = wi * drho + dphi + rho * wi * (T(3) * cu + T(4.5) * cu * cu - T(1.5) * usq);
    }

    if (P.collision == LBCG_BGK) {
#pragma unroll
        for (int i = 0; i < Q; ++i) g[i] = geq[i] + om1 * (g[i] - geq[i]);
    } else {
        T pxx = 0, pyy = 0, pzz = 0, pxy = 0, pxz = 0, pyz = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const T ne = g[i] - geq[i];
            const int ax = L::cx(i), ay = L::cy(i), az = L::cz(i);
            if (ax) pxx += ne;
            if (ay) pyy += ne;
            if (az) pzz += ne;
            if (ax && ay) pxy += (ax * ay > 0) ? ne : -ne;
            if (ax && az) pxz += (ax * az > 0) ? ne : -ne;
            if (ay && az) pyz += (ay * az > 0) ? ne : -ne;
        }
        const T third = T(1) / T(3);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int ax = L::cx(i), ay = L::cy(i), az = L::cz(i);
            T qp = ((T)(ax * ax) - third) * pxx + ((T)(ay * ay) - third) * pyy;
            if (L::D == 3) qp += ((T)(az * az) - third) * pzz;
            if (ax && ay) qp += T(2 * ax * ay) * pxy;
            if (ax && az) qp += T(2 * ax * az) * pxz;
            if (ay && az) qp += T(2 * ay * az) * pyz;
            g[i] = geq[i] + om1 * (T(4.5) * (T)L::w(i)) * qp;
        }
    }

    // perturbation (Eq. 9) and recolouring (Eq. 10)
    const T fn2 = F[0] * F[0] + F[1] * F[1] + F[2] * F[2];
    const bool has_f = fn2 > T(1e-20);
    const T fn = has_f ? sqrt(fn2) : T(0);
    const T inv_fn = has_f ? T(1) / fn : T(0);
    const T inv_fn2 = inv_fn * inv_fn;
    const T half_a_fn = T(0.5) * ph.A * fn;
    const T seg = ph.beta * rhoR * rhoB * inv_rho * inv_rho;
    const T fracR = rhoR * inv_rho;
    const T inv_sqrt2 = T(0.70710678118654752440);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T fc = (T)L::cx(i) * F[0] + (T)L::cy(i) * F[1] + (T)L::cz(i) * F[2];
        const T wi = (T)L::w(i);
        T gpost = g[i];
        if (has_f) gpost += half_a_fn * (wi * fc * fc * inv_fn2 - (T)L::Bc(i));
        const int c = L::cls(i);
        const T cosphi = (c == 0) ? T(0) : (c == 1 ? fc * inv_fn : fc * inv_fn * inv_sqrt2);
        const T e = rhoR * ph.phiR[c] + rhoB * ph.phiB[c];
        const T ftot = gpost + ph.wr0[c];
        r[i] = fracR * ftot + seg * cosphi * e;
        g[i] = gpost;
    }
}

}  // namespace lbcg
