// obs_kernels.cuh -- observable reductions (masses and momentum of Eqs. 2-3, the pressure
// of Eq. 8 in two windows, red amount, max |u|) shared by lbcg_observables and
// lbcg_observables_noalloc.  Per-site arithmetic runs in the storage format's compute
// type (FP64 only for FP64 storage: GB300's FP64 rate is low); per-thread and per-block
// accumulation is FP64.  Deterministic: a fixed grid, fixed per-thread site order, fixed
// shuffle/shared-memory trees, and one block combining the per-block rows in fixed order.
#pragma once

#include "lbcg_device.cuh"

namespace lbcg {
namespace {

// fluid-site predicates: library link words, or a caller's uint8 mask (code 0 = fluid)
struct FluidLink {
    const uint32_t* p;
    __device__ bool operator()(long long s) const { return !p || ((p[s] >> kTypeShift) & 3u) == kTypeFluid; }
};
struct FluidMask {
    const uint8_t* p;
    __device__ bool operator()(long long s) const { return !p || p[s] == LBCG_MASK_FLUID; }
};

constexpr int kObs1 = 8;  // mass_r, mass_b, mom x, y, z, red amount, max |u|, non-finite count
constexpr int kObs2 = 4;  // p_in sum, n_in, p_out sum, n_out

template <int NS>
__device__ __forceinline__ void obs_block_reduce(double (&v)[NS], unsigned maxmask, double* out_row)
{
    __shared__ double sh[32][NS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NS; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double t = __shfl_xor_sync(0xffffffffu, v[k], o);
            v[k] = ((maxmask >> k) & 1u) ? fmax(v[k], t) : v[k] + t;
        }
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NS; ++k) sh[warp][k] = v[k];
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            double t = lane < nw ? sh[lane][k] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double q = __shfl_xor_sync(0xffffffffu, t, o);
                t = ((maxmask >> k) & 1u) ? fmax(t, q) : t + q;
            }
            if (lane == 0) out_row[k] = t;
        }
    }
}

// moments of one site from the stored (post-collision) state, compute type T
template <int LAT, int PREC>
__device__ __forceinline__ void obs_site(const KParams& P, const typename Store<PREC>::S* __restrict__ a, size_t s,
                                         typename Store<PREC>::T& rr, typename Store<PREC>::T& rb,
                                         typename Store<PREC>::T& rho, typename Store<PREC>::T (&j)[3])
{
    using L = Lat<LAT>;
    using T = typename Store<PREC>::T;
    const Phys<T>& ph = phys<T>(P);
    T sg = 0;
    rr = 0;
    j[0] = j[1] = j[2] = 0;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        T r, g;
        Store<PREC>::load(a, (size_t)i * P.np + s, (size_t)(L::Q + i) * P.np + s, ph, L::cls(i), r, g);
        rr += r;
        sg += g;
        if (L::cx(i)) j[0] += L::cx(i) > 0 ? g : -g;
        if (L::cy(i)) j[1] += L::cy(i) > 0 ? g : -g;
        if (L::cz(i)) j[2] += L::cz(i) > 0 ? g : -g;
    }
    rho = ph.rho0 + sg;
    rb = rho - rr;
}

template <int LAT, int PREC, class FL>
__global__ void __launch_bounds__(256) k_obs1(const KParams P, const typename Store<PREC>::S* __restrict__ a,
                                              FL fluid, long long n, double* __restrict__ partials)
{
    using T = typename Store<PREC>::T;
    double v[kObs1] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x) {
        if (!fluid(s)) continue;
        T rr, rb, rho, j[3];
        obs_site<LAT, PREC>(P, a, (size_t)s, rr, rb, rho, j);
        if (!(rho > T(0)) || !isfinite(rho)) {
            v[7] += 1.0;
            continue;
        }
        v[0] += (double)rr;
        v[1] += (double)rb;
        v[2] += (double)j[0];
        v[3] += (double)j[1];
        v[4] += (double)j[2];
        v[5] += (double)((T(1) + (rr - rb) / rho) / T(2));
        v[6] = fmax(v[6], (double)(sqrt(j[0] * j[0] + j[1] * j[1] + j[2] * j[2]) / rho));
    }
    obs_block_reduce<kObs1>(v, 1u << 6, partials + (size_t)blockIdx.x * kObsSlots);
}

template <int LAT, int PREC, class FL>
__global__ void __launch_bounds__(256) k_obs2(const KParams P, const typename Store<PREC>::S* __restrict__ a,
                                              FL fluid, long long n, double cx, double cy, double cz, double kpr,
                                              double kpb, const double* __restrict__ res,
                                              double* __restrict__ partials)
{
    using L = Lat<LAT>;
    using T = typename Store<PREC>::T;
    const T r_in = (T)res[9], r_out = (T)res[10];
    const T tcx = (T)cx, tcy = (T)cy, tcz = (T)cz;
    const T tnx = (T)P.nx, tny = (T)P.ny, tnz = (T)P.nz;
    double v[kObs2] = {0, 0, 0, 0};
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x) {
        if (!fluid(s)) continue;
        const int x = (int)(s % P.nx);
        const int y = (int)((s / P.nx) % P.ny);
        const int z = (int)(s / ((long long)P.nx * P.ny));
        T d2 = 0, dd;
        dd = fabs((T)x - tcx);
        if (P.per[0] && tnx - dd < dd) dd = tnx - dd;
        d2 += dd * dd;
        dd = fabs((T)y - tcy);
        if (P.per[1] && tny - dd < dd) dd = tny - dd;
        d2 += dd * dd;
        if (L::D == 3) {
            dd = fabs((T)z - tcz);
            if (P.per[2] && tnz - dd < dd) dd = tnz - dd;
            d2 += dd * dd;
        }
        const T r = sqrt(d2);
        if (r >= r_in && r <= r_out) continue;
        T rr, rb, rho, j[3];
        obs_site<LAT, PREC>(P, a, (size_t)s, rr, rb, rho, j);
        const double p = kpr * (double)rr + kpb * (double)rb;
        if (r < r_in) {
            v[0] += p;
            v[1] += 1.0;
        } else {
            v[2] += p;
            v[3] += 1.0;
        }
    }
    obs_block_reduce<kObs2>(v, 0u, partials + (size_t)blockIdx.x * kObsSlots);
}

// one block of 256 threads: rows nb of ns slots combined in fixed order into res[off..]
__global__ void __launch_bounds__(256) k_obs_fin(const double* __restrict__ partials, int nb, int ns,
                                                 unsigned maxmask, int off, double* __restrict__ res, int dim,
                                                 double r_in, double r_out)
{
    __shared__ double sh[8][kObsSlots];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < ns; ++k) {
        const bool mx = (maxmask >> k) & 1u;
        double t = 0.0;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            const double q = partials[(size_t)b * kObsSlots + k];
            t = mx ? fmax(t, q) : t + q;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double q = __shfl_xor_sync(0xffffffffu, t, o);
            t = mx ? fmax(t, q) : t + q;
        }
        if (lane == 0) sh[warp][k] = t;
    }
    __syncthreads();
    if ((int)threadIdx.x < ns) {
        const int k = threadIdx.x;
        const bool mx = (maxmask >> k) & 1u;
        double t = sh[0][k];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) t = mx ? fmax(t, sh[w][k]) : t + sh[w][k];
        res[off + k] = t;
    }
    __syncthreads();
    if (off == 0 && threadIdx.x == 0) {
        const double pi = 3.14159265358979323846;
        const double reff = dim == 2 ? sqrt(res[5] / pi) : cbrt(3.0 * res[5] / (4.0 * pi));
        res[8] = reff;
        res[9] = r_in < 0.0 ? reff / 2.0 : r_in;
        res[10] = r_out < 0.0 ? reff + 5.0 : r_out;
    }
}

// the whole observable sequence on one stream: pass 1, combine (+ radius and windows),
// pass 2, combine; results in res[0..15) (layout of lbcg_obs assembly in the callers)
template <class FL>
cudaError_t run_observables(const lbcg_ctx& c, const void* a, FL fluid, const double centre[3], double r_in,
                            double r_out, int nb, double* partials, double* res, cudaStream_t st)
{
    const int dim = c.D;
    const double kpr = dim == 2 ? 3.0 * (1.0 - c.p.alpha_r) / 5.0 : (1.0 - c.p.alpha_r) / 2.0;
    const double kpb = dim == 2 ? 3.0 * (1.0 - c.p.alpha_b) / 5.0 : (1.0 - c.p.alpha_b) / 2.0;
    const KParams& P = c.kp;
    const long long n = c.n;
#define OBS_DISPATCH(F)                                                        \
    do {                                                                       \
        const int prec_ = c.p.precision;                                      \
        if (c.p.lattice == LBCG_D2Q9) {                                        \
            if (prec_ == LBCG_FP64) F(0, LBCG_FP64);                           \
            else if (prec_ == LBCG_FP32) F(0, LBCG_FP32);                      \
            else if (prec_ == LBCG_FP32_DEV) F(0, LBCG_FP32_DEV);              \
            else F(0, LBCG_FP16_SCALED);                                       \
        } else {                                                               \
            if (prec_ == LBCG_FP64) F(1, LBCG_FP64);                           \
            else if (prec_ == LBCG_FP32) F(1, LBCG_FP32);                      \
            else if (prec_ == LBCG_FP32_DEV) F(1, LBCG_FP32_DEV);              \
            else F(1, LBCG_FP16_SCALED);                                       \
        }                                                                      \
    } while (0)
#define OBS1_(LAT, PREC) \
    k_obs1<LAT, PREC, FL><<<nb, 256, 0, st>>>(P, (const typename Store<PREC>::S*)a, fluid, n, partials)
#define OBS2_(LAT, PREC)                                                                                    \
    k_obs2<LAT, PREC, FL><<<nb, 256, 0, st>>>(P, (const typename Store<PREC>::S*)a, fluid, n, centre[0],   \
                                              centre[1], centre[2], kpr, kpb, res, partials)
    OBS_DISPATCH(OBS1_);
    k_obs_fin<<<1, 256, 0, st>>>(partials, nb, kObs1, 1u << 6, 0, res, dim, r_in, r_out);
    OBS_DISPATCH(OBS2_);
    k_obs_fin<<<1, 256, 0, st>>>(partials, nb, kObs2, 0u, 11, res, dim, r_in, r_out);
#undef OBS1_
#undef OBS2_
#undef OBS_DISPATCH
    return cudaGetLastError();
}

}  // namespace
}  // namespace lbcg
