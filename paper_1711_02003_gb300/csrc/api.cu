// api.cu -- host side of the C ABI declared in include/lbcg.h: parameter checks,
// geometry preprocessing (link words, port ghost tables, inlet profiles), buffer
// binding, step sequencing and synchronous read-back.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "lbcg_device.cuh"

using namespace lbcg;

namespace {

thread_local std::string g_err = "no error";

int fail(int code, const std::string& msg)
{
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* where)
{
    g_err = std::string(where) + ": " + cudaGetErrorString(e);
    return LBCG_ERR_CUDA;
}

#define LBCG_CUDA(call, where)                          \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

int q_of(int lattice) { return lattice == LBCG_D2Q9 ? 9 : 19; }

long long sites_of(const lbcg_params* p)
{
    return (long long)p->nx * p->ny * (p->lattice == LBCG_D2Q9 ? 1 : p->nz);
}

int validate(const lbcg_params* p)
{
    if (!p) return fail(LBCG_ERR_ARG, "null parameters");
    if (p->lattice != LBCG_D2Q9 && p->lattice != LBCG_D3Q19) return fail(LBCG_ERR_ARG, "unknown lattice");
    if (p->precision < LBCG_FP64 || p->precision > LBCG_FP16_SCALED) return fail(LBCG_ERR_ARG, "unknown precision");
    if (p->collision != LBCG_REG && p->collision != LBCG_BGK) return fail(LBCG_ERR_ARG, "unknown collision");
    if (p->nx < 1 || p->ny < 1 || (p->lattice == LBCG_D3Q19 && p->nz < 1))
        return fail(LBCG_ERR_ARG, "box sizes must be >= 1");
    const long long n = sites_of(p);
    if (n > (long long)INT32_MAX - 1) return fail(LBCG_ERR_ARG, "more than 2^31-2 sites");
    if (!(p->tau_r > 0.5) || !(p->tau_b > 0.5)) return fail(LBCG_ERR_ARG, "relaxation times must exceed 1/2");
    if (!(p->beta >= 0.0 && p->beta <= 1.0)) return fail(LBCG_ERR_ARG, "beta must lie in [0,1]");
    if (!(p->A >= 0.0) || !std::isfinite(p->A)) return fail(LBCG_ERR_ARG, "A must be finite and >= 0");
    if (!(p->alpha_r > 0.0 && p->alpha_r < 1.0) || !(p->alpha_b > 0.0 && p->alpha_b < 1.0))
        return fail(LBCG_ERR_ARG, "alpha_k must lie in (0,1)");
    if (!(p->rho0 > 0.0) || !std::isfinite(p->rho0)) return fail(LBCG_ERR_ARG, "rho0 must be > 0");
    if (!(p->psi_wall >= -1.0 && p->psi_wall <= 1.0)) return fail(LBCG_ERR_ARG, "psi_wall must lie in [-1,1]");
    return LBCG_OK;
}

size_t elem_size(int precision)
{
    switch (precision) {
        case LBCG_FP64: return 8;
        case LBCG_FP32:
        case LBCG_FP32_DEV: return 4;
        default: return 2;
    }
}

size_t padded(long long n) { return (size_t)((n + 127) / 128 * 128); }

// lattice velocity sets in the ABI order, for host-side geometry work
void host_c(int lattice, int i, int c[3])
{
    if (lattice == LBCG_D2Q9) {
        c[0] = Lat<0>::cx(i);
        c[1] = Lat<0>::cy(i);
        c[2] = 0;
    } else {
        c[0] = Lat<1>::cx(i);
        c[1] = Lat<1>::cy(i);
        c[2] = Lat<1>::cz(i);
    }
}

template <typename T>
void fill_phys(Phys<T>& ph, const lbcg_params& p, int lattice)
{
    const double nu_r = (p.tau_r - 0.5) / 3.0, nu_b = (p.tau_b - 0.5) / 3.0;
    const double w[3] = {lattice == 0 ? 4.0 / 9.0 : 1.0 / 3.0, lattice == 0 ? 1.0 / 9.0 : 1.0 / 18.0, 1.0 / 36.0};
    // Eq. 7 for D2Q9; D3Q19 uses alpha, (1-alpha)/12, (1-alpha)/24 (reduces to w_i at alpha = 1/3)
    const double d1 = lattice == 0 ? 5.0 : 12.0, d2 = lattice == 0 ? 20.0 : 24.0;
    const double phR[3] = {p.alpha_r, (1.0 - p.alpha_r) / d1, (1.0 - p.alpha_r) / d2};
    const double phB[3] = {p.alpha_b, (1.0 - p.alpha_b) / d1, (1.0 - p.alpha_b) / d2};
    ph.rho0 = (T)p.rho0;
    ph.half_inv_nu_r = (T)(0.5 / nu_r);
    ph.half_inv_nu_b = (T)(0.5 / nu_b);
    ph.A = (T)p.A;
    ph.beta = (T)p.beta;
    ph.psi_wall = (T)p.psi_wall;
    for (int c = 0; c < 3; ++c) {
        ph.phiR[c] = (T)phR[c];
        ph.phiB[c] = (T)phB[c];
        ph.dphiR[c] = (T)(phR[c] - w[c]);
        ph.dphiB[c] = (T)(phB[c] - w[c]);
        ph.wr0[c] = (T)(w[c] * p.rho0);
        ph.w[c] = (T)w[c];
        ph.inv_w[c] = (T)(1.0 / w[c]);
    }
    ph.scale_g = (T)256.0;
    ph.inv_scale_g = (T)(1.0 / 256.0);
}

}  // namespace

namespace lbcg {

size_t storage_size(int precision) { return elem_size(precision); }

KParams make_kparams(const lbcg_params& p, const int dims[3], size_t np, int rows_req, int block_rows)
{
    KParams k;
    std::memset(&k, 0, sizeof(k));
    k.nx = dims[0];
    k.ny = dims[1];
    k.nz = dims[2];
    for (int a = 0; a < 3; ++a) k.per[a] = p.periodic[a] ? 1 : 0;
    if (p.lattice == LBCG_D2Q9) k.per[2] = 1;
    k.np = np;
    k.collision = p.collision;
    k.lattice = p.lattice;
    k.alpha_r = p.alpha_r;
    k.alpha_b = p.alpha_b;
    fill_phys(k.pf, p, p.lattice);
    fill_phys(k.pd, p, p.lattice);
    const int sms = 152;
    if (p.lattice == LBCG_D2Q9) {
        // strips of 30 x rows sites per warp; rows trade the ring re-reads (2/rows) against
        // enough warps for about four waves of 24 resident warps per SM (measured best: 16-32)
        k.nsx = (k.nx + 29) / 30;
        int rows = rows_req;
        if (rows <= 0) {
            const long long target = (long long)sms * 24 * 4;
            long long r = ((long long)k.nsx * k.ny) / target;
            rows = (int)std::max(4LL, std::min(32LL, r));
        }
        k.rows = std::min(rows, k.ny);
        k.nsy = (k.ny + k.rows - 1) / k.rows;
        k.nsz = 1;
    } else {
        // blocks of 32 x 8 threads marching 8 z-planes (measured best)
        const int wy = block_rows > 2 ? block_rows : 8;
        k.nsx = (k.nx + 29) / 30;
        k.nsy = (k.ny + (wy - 2) - 1) / (wy - 2);
        const int rows = rows_req > 0 ? rows_req : 8;
        k.rows = std::min(rows, k.nz);
        k.nsz = (k.nz + k.rows - 1) / k.rows;
    }
    return k;
}

void fill_kparams(lbcg_ctx* c)
{
    if (c->p.lattice != LBCG_D2Q9 && c->block_rows <= 2) c->block_rows = 8;
    c->kp = make_kparams(c->p, c->dims, c->np, c->rows, c->block_rows);
    c->kp.stall_test = c->stall_test;
    c->kp.status = c->d_status;
    c->kp.ntiles = c->d_tiles ? c->ntiles : 0;
}

// active-tile list of the current launch shape (walled geometries): tiles (2D strips of
// 30 x rows, 3D blocks of 30 x (block_rows-2) x rows) holding at least one fluid site
// D3Q19 block tiles of launch shape k (30 x ty sites per x-y column) that hold fluid:
// for each column, the planes holding a fluid site grouped in runs of consecutive planes,
// each run cut into near-equal z-ranges of at most k.rows planes (a terrace 8 planes high
// gets two ranges of 4, not a range of 4 and one of 4 holding one fluid plane).  Appends
// (column index, z0 | z1 << 16) pairs ordered by range, then column.  False if nz > 65535.
bool fitted_tiles_3d(const lbcg_ctx* c, const KParams& k, int ty, std::vector<int>& list)
{
    const int nx = c->dims[0], ny = c->dims[1], nz = c->dims[2];
    if (nz > 0xffff) return false;
    const long long ncol = (long long)k.nsx * k.nsy;
    std::vector<char> has((size_t)(ncol * nz), 0);
    for (long long s = 0; s < c->n; ++s) {
        if (c->mask[s] != LBCG_MASK_FLUID) continue;
        const int x = (int)(s % nx), y = (int)((s / nx) % ny), z = (int)(s / ((long long)nx * ny));
        has[(size_t)(((x / 30) + (long long)k.nsx * (y / ty)) * nz + z)] = 1;
    }
    std::vector<std::vector<std::pair<int, int>>> ranges((size_t)ncol);
    size_t depth = 0;
    for (long long col = 0; col < ncol; ++col) {
        const char* h = &has[(size_t)(col * nz)];
        for (int z = 0; z < nz;) {
            if (!h[z]) {
                ++z;
                continue;
            }
            int e = z;
            while (e < nz && h[e]) ++e;
            const int len = e - z, parts = (len + k.rows - 1) / k.rows;
            for (int q = 0; q < parts; ++q)
                ranges[(size_t)col].push_back(
                    {z + (int)((long long)len * q / parts), z + (int)((long long)len * (q + 1) / parts)});
            z = e;
        }
        depth = std::max(depth, ranges[(size_t)col].size());
    }
    for (size_t d = 0; d < depth; ++d)
        for (long long col = 0; col < ncol; ++col)
            if (d < ranges[(size_t)col].size()) {
                list.push_back((int)col);
                list.push_back(ranges[(size_t)col][d].first | (ranges[(size_t)col][d].second << 16));
            }
    return true;
}

static int build_active_tiles(lbcg_ctx* c);

int build_tiles(lbcg_ctx* c)
{
    return build_active_tiles(c);
}

// the per-tile row lists (gstart, grow) of the fused port refill from owner[g], the active-tile
// index whose sites include ghost g's inward neighbour x'
static int upload_tile_ghosts(lbcg_ctx* c, int nt, const std::vector<int>& owner)
{
    std::vector<int> count((size_t)nt + 1, 0);
    for (int g = 0; g < c->nghost; ++g) ++count[(size_t)owner[(size_t)g] + 1];
    for (int t = 0; t < nt; ++t) count[(size_t)t + 1] += count[(size_t)t];
    std::vector<int> rows((size_t)std::max(c->nghost, 1)), fillp(count.begin(), count.end() - 1);
    for (int g = 0; g < c->nghost; ++g) rows[(size_t)fillp[(size_t)owner[(size_t)g]]++] = g;
    if (cudaMalloc(&c->d_gstart, sizeof(int) * count.size()) != cudaSuccess ||
        cudaMalloc(&c->d_grow, sizeof(int) * rows.size()) != cudaSuccess)
        return fail(LBCG_ERR_NOMEM, "tile ghost list allocation failed");
    if (cudaMemcpy(c->d_gstart, count.data(), sizeof(int) * count.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->d_grow, rows.data(), sizeof(int) * rows.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(LBCG_ERR_CUDA, "tile ghost list copy failed");
    return LBCG_OK;
}

// D3Q19 tiles of list `list` (column, z0 | z1 << 16): for every port ghost the tile that
// collides its x', as per-tile row lists (gstart, grow) for the fused refill of the moment marches
static int build_tile_ghosts(lbcg_ctx* c, const std::vector<int>& list)
{
    const KParams& k = c->kp;
    const int nx = c->dims[0], ny = c->dims[1], ty = c->block_rows - 2;
    const int nt = (int)(list.size() / 2);
    std::vector<std::vector<int>> by_col((size_t)k.nsx * k.nsy);
    for (int t = 0; t < nt; ++t) by_col[(size_t)list[2 * t]].push_back(t);
    std::vector<int> owner((size_t)c->nghost, -1);
    for (int g = 0; g < c->nghost; ++g) {
        const long long s = c->ghost_xp[(size_t)g];
        const int x = (int)(s % nx), y = (int)((s / nx) % ny), z = (int)(s / ((long long)nx * ny));
        for (int t : by_col[(size_t)((x / 30) + (long long)k.nsx * (y / ty))]) {
            const int z0 = list[2 * t + 1] & 0xffff, z1 = list[2 * t + 1] >> 16;
            if (z >= z0 && z < z1) owner[(size_t)g] = t;
        }
        if (owner[(size_t)g] < 0) return fail(LBCG_ERR_GEOMETRY, "a port's inward neighbour lies in no tile");
    }
    return upload_tile_ghosts(c, nt, owner);
}

// D2Q9 strips of list `list` (strip index sx + nsx sy): for every port ghost the strip whose
// warp collides its x', for the fused refill of the strip marches
static int build_strip_ghosts(lbcg_ctx* c, const std::vector<int>& list)
{
    const KParams& k = c->kp;
    const int nx = c->dims[0];
    const int nt = (int)list.size();
    std::vector<int> index((size_t)k.nsx * k.nsy, -1);
    for (int t = 0; t < nt; ++t) index[(size_t)list[(size_t)t]] = t;
    std::vector<int> owner((size_t)c->nghost, -1);
    for (int g = 0; g < c->nghost; ++g) {
        const long long s = c->ghost_xp[(size_t)g];
        const int x = (int)(s % nx), y = (int)(s / nx);
        owner[(size_t)g] = index[(size_t)((x / 30) + (long long)k.nsx * (y / k.rows))];
        if (owner[(size_t)g] < 0) return fail(LBCG_ERR_GEOMETRY, "a port's inward neighbour lies in no strip");
    }
    return upload_tile_ghosts(c, nt, owner);
}

static int build_active_tiles(lbcg_ctx* c)
{
    cudaFree(c->d_tiles);
    cudaFree(c->d_gstart);
    cudaFree(c->d_grow);
    c->d_tiles = nullptr;
    c->d_gstart = nullptr;
    c->d_grow = nullptr;
    c->ntiles = 0;
    c->kp.ntiles = 0;
    if (!c->geometry || !c->any_link) return LBCG_OK;
    const KParams& k = c->kp;
    const int nx = c->dims[0], ny = c->dims[1], nz = c->dims[2];
    std::vector<int> list;
    if (c->p.lattice == LBCG_D2Q9) {
        // strips of 30 x rows sites holding a fluid site
        const long long ntot = (long long)k.nsx * k.nsy;
        std::vector<char> on((size_t)ntot, 0);
        for (long long s = 0; s < c->n; ++s) {
            if (c->mask[s] != LBCG_MASK_FLUID) continue;
            const int x = (int)(s % nx), y = (int)(s / nx);
            on[(size_t)((x / 30) + (long long)k.nsx * (y / k.rows))] = 1;
        }
        for (long long t = 0; t < ntot; ++t)
            if (on[(size_t)t]) list.push_back((int)t);
        if ((long long)list.size() == ntot && c->nghost == 0) return LBCG_OK;  // nothing to skip
        if (list.empty()) list.push_back(0);
    } else {
        if (!fitted_tiles_3d(c, k, c->block_rows - 2, list)) return fail(LBCG_ERR_GEOMETRY, "nz above 65535 with walls");
        if (list.empty()) {
            list.push_back(0);
            list.push_back(0);  // an empty range: the block pulls ring planes only
        }
    }
    if (cudaMalloc(&c->d_tiles, sizeof(int) * list.size()) != cudaSuccess)
        return fail(LBCG_ERR_NOMEM, "tile list allocation failed");
    if (cudaMemcpy(c->d_tiles, list.data(), sizeof(int) * list.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(LBCG_ERR_CUDA, "tile list copy failed");
    c->ntiles = (int)(c->p.lattice == LBCG_D2Q9 ? list.size() : list.size() / 2);
    c->kp.ntiles = c->ntiles;
    if (c->nghost > 0) return c->p.lattice == LBCG_D3Q19 ? build_tile_ghosts(c, list) : build_strip_ghosts(c, list);
    return LBCG_OK;
}

}  // namespace lbcg

extern "C" {
static void drop_graphs(lbcg_ctx* c);
}

static void free_tables(lbcg_ctx* c)
{
    cudaFree(c->d_link);
    cudaFree(c->d_ghost);
    cudaFree(c->d_ghost_u);
    cudaFree(c->d_gpsi);
    c->d_link = nullptr;
    c->d_ghost = nullptr;
    c->d_ghost_u = nullptr;
    c->d_gpsi = nullptr;
    c->gpsi_buf[0] = c->gpsi_buf[1] = nullptr;
}

namespace lbcg {

// The table of a buffer stays with it while it is one of the two state buffers; a buffer
// met for the first time (first use, or new buffers bound) takes a table whose buffer is no
// longer a state buffer.  Every step reads the table of its input only after a refill of
// that buffer's ghosts wrote it (the refill launch, or the previous step's fused refill).
void* gpsi_for(lbcg_ctx* c, const void* buf)
{
    if (!c->d_gpsi || !buf) return nullptr;
    for (int k = 0; k < 2; ++k)
        if (c->gpsi_buf[k] == buf) return c->d_gpsi + (size_t)k * c->nghost;
    for (int k = 0; k < 2; ++k)
        if (c->gpsi_buf[k] != c->A && c->gpsi_buf[k] != c->B) {
            c->gpsi_buf[k] = buf;
            return c->d_gpsi + (size_t)k * c->nghost;
        }
    return nullptr;
}

}  // namespace lbcg

extern "C" {

const char* lbcg_strerror(int s)
{
    switch (s) {
        case LBCG_OK: return "ok";
        case LBCG_ERR_ARG: return "invalid argument";
        case LBCG_ERR_STATE: return "call out of order";
        case LBCG_ERR_CUDA: return "CUDA error";
        case LBCG_ERR_NOMEM: return "out of device memory";
        case LBCG_ERR_DIVERGED: return "non-finite or non-positive density";
        case LBCG_ERR_GEOMETRY: return "invalid geometry";
        case LBCG_ERR_CAPACITY: return "output capacity too small";
        case LBCG_ERR_UNSUPPORTED: return "unsupported";
        case LBCG_ERR_TIMEOUT: return "bounded wait or iteration ran out";
        case LBCG_ERR_BOUNDS: return "index outside its array (bounds-checked build)";
        default: return "unknown status";
    }
}

const char* lbcg_last_error(void) { return g_err.c_str(); }

int lbcg_abi_version(void) { return LBCG_ABI_VERSION; }

int lbcg_bounds_checked(void)
{
#ifdef LBCG_CHECK_BOUNDS
    return 1;
#else
    return 0;
#endif
}

int lbcg_fma_peak(int precision, void* stream, double* gflops)
{
    std::string err;
    const int st = lbcg::fma_peak(precision, stream, gflops, err);
    return st ? fail(st, err) : LBCG_OK;
}

size_t lbcg_state_bytes(const lbcg_params* p)
{
    if (validate(p) != LBCG_OK) return 0;
    return (size_t)2 * q_of(p->lattice) * padded(sites_of(p)) * elem_size(p->precision);
}

int lbcg_create(const lbcg_params* p, void* stream, lbcg_ctx** out)
{
    if (!out) return fail(LBCG_ERR_ARG, "null output pointer");
    *out = nullptr;
    int st = validate(p);
    if (st) return st;
    lbcg_ctx* c = new (std::nothrow) lbcg_ctx();
    if (!c) return fail(LBCG_ERR_NOMEM, "host allocation failed");
    c->p = *p;
    if (c->p.lattice == LBCG_D2Q9) c->p.nz = 1;
    c->stream = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "cudaGetDevice");
    }
    c->Q = q_of(c->p.lattice);
    c->D = c->p.lattice == LBCG_D2Q9 ? 2 : 3;
    c->dims[0] = c->p.nx;
    c->dims[1] = c->p.ny;
    c->dims[2] = c->p.nz;
    c->n = sites_of(&c->p);
    c->np = padded(c->n);
    c->state_bytes = (size_t)2 * c->Q * c->np * elem_size(c->p.precision);
    {
        const char* t = std::getenv("LBCG_TEST_PIPELINE_STALL");
        c->stall_test = t && t[0] == '1';
    }
    fill_kparams(c);
    // status word of the bounded pipeline waits in the TMA-staged step kernel
    if (cudaMalloc(&c->d_status, sizeof(int)) != cudaSuccess || cudaMemset(c->d_status, 0, sizeof(int)) != cudaSuccess) {
        cudaFree(c->d_status);
        delete c;
        return fail(LBCG_ERR_NOMEM, "status word allocation failed");
    }
    *out = c;
    return LBCG_OK;
}

void lbcg_destroy(lbcg_ctx* c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    free_tables(c);
    cudaFree(c->d_tiles);
    cudaFree(c->d_gstart);
    cudaFree(c->d_grow);
    cudaFree(c->d_scratch);
    cudaFree(c->d_partials);
    cudaFree(c->d_result);
    cudaFree(c->d_status);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    delete c;
}

int lbcg_bind_state(lbcg_ctx* c, void* a, void* b, size_t bytes)
{
    if (!c || !a || !b) return fail(LBCG_ERR_ARG, "null context or buffer");
    if (a == b) return fail(LBCG_ERR_ARG, "the two state buffers must differ");
    if (bytes < c->state_bytes) return fail(LBCG_ERR_ARG, "state buffers smaller than lbcg_state_bytes");
    if (((uintptr_t)a | (uintptr_t)b) & 255u) return fail(LBCG_ERR_ARG, "state buffers must be 256-byte aligned");
    drop_graphs(c);
    c->A = a;
    c->B = b;
    c->bound = true;
    c->fields = false;
    c->ghosts_fresh = false;
    return LBCG_OK;
}

int lbcg_set_geometry(lbcg_ctx* c, const uint8_t* mask, const lbcg_port* ports, int nports)
{
    if (!c || !mask) return fail(LBCG_ERR_ARG, "null context or mask");
    if (nports < 0 || nports > LBCG_MAX_PORTS || (nports > 0 && !ports))
        return fail(LBCG_ERR_ARG, "port count out of range");
    const int nx = c->dims[0], ny = c->dims[1], nz = c->dims[2];
    const long long n = c->n;
    const int Q = c->Q;
    int per[3] = {c->p.periodic[0] ? 1 : 0, c->p.periodic[1] ? 1 : 0, c->p.periodic[2] ? 1 : 0};
    if (c->p.lattice == LBCG_D2Q9) per[2] = 1;
    for (int m = 0; m < nports; ++m) {
        const lbcg_port& pt = ports[m];
        if (pt.kind < 0 || pt.kind > 2) return fail(LBCG_ERR_GEOMETRY, "unknown port kind");
        if (pt.normal_axis < 0 || pt.normal_axis >= c->D || (pt.normal_sign != 1 && pt.normal_sign != -1))
            return fail(LBCG_ERR_GEOMETRY, "bad port normal");
        if (!(pt.psi >= -1.0 && pt.psi <= 1.0) || !(pt.rho > 0.0) || !std::isfinite(pt.u_max))
            return fail(LBCG_ERR_GEOMETRY, "bad port values");
    }
    std::vector<uint32_t> link((size_t)n);
    bool any = false;
    long long fluid = 0;
    int lo[LBCG_MAX_PORTS][3], hi[LBCG_MAX_PORTS][3];
    for (int m = 0; m < LBCG_MAX_PORTS; ++m)
        for (int a = 0; a < 3; ++a) {
            lo[m][a] = 1 << 30;
            hi[m][a] = -1;
        }
    std::vector<long long> ghosts;
    auto at = [&](long long x, long long y, long long z) { return x + (long long)nx * (y + (long long)ny * z); };
    for (long long s = 0; s < n; ++s) {
        const int code = mask[s];
        const int x = (int)(s % nx), y = (int)((s / nx) % ny), z = (int)(s / ((long long)nx * ny));
        if (code == LBCG_MASK_WALL) {
            link[s] = kTypeWall << kTypeShift;
            any = true;
            continue;
        }
        if (code >= LBCG_MASK_PORT0) {
            const int m = code - LBCG_MASK_PORT0;
            if (m >= nports) return fail(LBCG_ERR_GEOMETRY, "mask names a port beyond nports");
            link[s] = kTypePort << kTypeShift;
            any = true;
            int v[3] = {x, y, z};
            for (int a = 0; a < 3; ++a) {
                lo[m][a] = std::min(lo[m][a], v[a]);
                hi[m][a] = std::max(hi[m][a], v[a]);
            }
            v[ports[m].normal_axis] += ports[m].normal_sign;
            const int dims[3] = {nx, ny, nz};
            const int ax = ports[m].normal_axis;
            if (v[ax] < 0 || v[ax] >= dims[ax] || mask[at(v[0], v[1], v[2])] != LBCG_MASK_FLUID)
                return fail(LBCG_ERR_GEOMETRY, "a port ghost's inward neighbour is not a fluid site");
            ghosts.push_back(s);
            continue;
        }
        if (code != LBCG_MASK_FLUID) return fail(LBCG_ERR_GEOMETRY, "unknown mask code");
        ++fluid;
        uint32_t lk = 0;
        for (int i = 1; i < Q; ++i) {
            int cc[3];
            host_c(c->p.lattice, i, cc);
            int v[3] = {x - cc[0], y - cc[1], z - cc[2]};
            const int dims[3] = {nx, ny, nz};
            bool out = false;
            for (int a = 0; a < 3; ++a) {
                if (v[a] < 0 || v[a] >= dims[a]) {
                    if (!per[a]) out = true;
                    v[a] = (v[a] + dims[a]) % dims[a];
                }
            }
            if (out || mask[at(v[0], v[1], v[2])] == LBCG_MASK_WALL) lk |= 1u << i;
        }
        if (lk) any = true;
        link[s] = lk;
    }
    // ghost table: [site | inward neighbour | port | kind] and [ux | uy | uz | rho | psi]
    const int ng = (int)ghosts.size();
    // the port site's link word carries its ghost-table row (the ghost-psi table)
    const bool gpsi = ng > 0 && (long long)ng <= (long long)kGhostMask + 1;
    if (gpsi)
        for (int t = 0; t < ng; ++t) link[(size_t)ghosts[t]] |= (uint32_t)t;
    std::vector<int> tab((size_t)4 * std::max(ng, 1));
    std::vector<double> gu((size_t)5 * std::max(ng, 1));
    for (int t = 0; t < ng; ++t) {
        const long long s = ghosts[t];
        const int m = mask[s] - LBCG_MASK_PORT0;
        const lbcg_port& pt = ports[m];
        int v[3] = {(int)(s % nx), (int)((s / nx) % ny), (int)(s / ((long long)nx * ny))};
        int w3[3] = {v[0], v[1], v[2]};
        w3[pt.normal_axis] += pt.normal_sign;
        tab[t] = (int)s;
        tab[ng + t] = (int)at(w3[0], w3[1], w3[2]);
        tab[2 * ng + t] = m;
        tab[3 * ng + t] = pt.kind;
        // parabolic (or flat) profile over the port's transverse extent, walls halfway
        double mag = pt.u_max;
        if (pt.profile == LBCG_PROFILE_PARABOLIC) {
            for (int a = 0; a < c->D; ++a) {
                if (a == pt.normal_axis) continue;
                const double W = (double)(hi[m][a] - lo[m][a] + 1);
                const double sc = (double)(v[a] - lo[m][a]) + 0.5;
                mag *= 4.0 * sc * (W - sc) / (W * W);
            }
        }
        double u[3] = {0.0, 0.0, 0.0};
        u[pt.normal_axis] = mag * pt.normal_sign;
        gu[t] = u[0];
        gu[ng + t] = u[1];
        gu[2 * ng + t] = u[2];
        gu[3 * ng + t] = pt.rho;
        gu[4 * ng + t] = pt.psi;
    }
    drop_graphs(c);
    free_tables(c);
    if (cudaMalloc(&c->d_link, sizeof(uint32_t) * (size_t)n) != cudaSuccess)
        return fail(LBCG_ERR_NOMEM, "link table allocation failed");
    if (ng > 0) {
        if (cudaMalloc(&c->d_ghost, sizeof(int) * tab.size()) != cudaSuccess ||
            cudaMalloc(&c->d_ghost_u, sizeof(double) * gu.size()) != cudaSuccess ||
            (gpsi && cudaMalloc(&c->d_gpsi, sizeof(double) * 2 * (size_t)ng) != cudaSuccess)) {
            free_tables(c);
            return fail(LBCG_ERR_NOMEM, "port table allocation failed");
        }
    }
    if (!c->d_partials) {
        if (cudaMalloc(&c->d_partials, sizeof(double) * kMaxPartials * kObsSlots) != cudaSuccess ||
            cudaMalloc(&c->d_result, sizeof(double) * 2 * kObsSlots) != cudaSuccess) {
            free_tables(c);
            return fail(LBCG_ERR_NOMEM, "reduction scratch allocation failed");
        }
    }
    LBCG_CUDA(cudaMemcpyAsync(c->d_link, link.data(), sizeof(uint32_t) * (size_t)n, cudaMemcpyHostToDevice,
                              c->stream),
              "copy link table");
    if (ng > 0) {
        LBCG_CUDA(cudaMemcpyAsync(c->d_ghost, tab.data(), sizeof(int) * tab.size(), cudaMemcpyHostToDevice,
                                  c->stream),
                  "copy ghost table");
        LBCG_CUDA(cudaMemcpyAsync(c->d_ghost_u, gu.data(), sizeof(double) * gu.size(), cudaMemcpyHostToDevice,
                                  c->stream),
                  "copy ghost velocities");
    }
    LBCG_CUDA(cudaStreamSynchronize(c->stream), "set_geometry sync");
    c->mask.assign(mask, mask + n);
    c->nports = nports;
    for (int m = 0; m < nports; ++m) c->ports[m] = ports[m];
    c->nghost = ng;
    c->ghost_xp.assign(tab.begin() + ng, tab.begin() + 2 * ng);
    c->any_link = any;
    c->fluid_sites = fluid;
    c->geometry = true;
    c->fields = false;
    c->ghosts_fresh = false;
    fill_kparams(c);
    return build_tiles(c);
}

// device scratch of at least `bytes` for staging and read-back (never the state buffers,
// so the stored state stays defined at every site)
static int scratch(lbcg_ctx* c, size_t bytes, void** out)
{
    if (c->scratch_bytes < bytes) {
        if (c->d_scratch) {
            cudaError_t e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) return cuda_fail(e, "scratch sync");
            cudaFree(c->d_scratch);
            c->d_scratch = nullptr;
            c->scratch_bytes = 0;
        }
        if (cudaMalloc(&c->d_scratch, bytes) != cudaSuccess) return fail(LBCG_ERR_NOMEM, "scratch allocation failed");
        c->scratch_bytes = bytes;
    }
    *out = c->d_scratch;
    return LBCG_OK;
}

// after A has been (re)initialised: give B the same contents, so both buffers hold a
// defined value at every site (walls stay zero, ghosts are refilled each step)
static int mirror_state(lbcg_ctx* c)
{
    c->ghosts_fresh = false;
    LBCG_CUDA(cudaMemcpyAsync(c->B, c->A, c->state_bytes, cudaMemcpyDeviceToDevice, c->stream), "mirror state");
    return LBCG_OK;
}

static int need(lbcg_ctx* c, bool fields)
{
    if (!c) return fail(LBCG_ERR_ARG, "null context");
    if (!c->bound) return fail(LBCG_ERR_STATE, "no state buffers bound");
    if (!c->geometry) return fail(LBCG_ERR_STATE, "no geometry set");
    if (fields && !c->fields) return fail(LBCG_ERR_STATE, "no initial fields set");
    return LBCG_OK;
}

int lbcg_init_fields_device(lbcg_ctx* c, const double* rr, const double* rb, const double* u)
{
    int st = need(c, false);
    if (st) return st;
    if (!rr || !rb) return fail(LBCG_ERR_ARG, "null density field");
    LBCG_CUDA(launch_init(c, rr, rb, u, c->A), "init kernel");
    st = mirror_state(c);
    if (st) return st;
    c->fields = true;
    c->step = 0;
    return LBCG_OK;
}

int lbcg_init_fields(lbcg_ctx* c, const double* rr, const double* rb, const double* u)
{
    const lbcg::TraceRange trace("lbcg_init_fields");
    int st = need(c, false);
    if (st) return st;
    if (!rr || !rb) return fail(LBCG_ERR_ARG, "null density field");
    // staging: rho_r | rho_b | u
    const size_t n = (size_t)c->n;
    void* sp = nullptr;
    st = scratch(c, n * 8 * (2 + c->D), &sp);
    if (st) return st;
    double* stg = (double*)sp;
    LBCG_CUDA(cudaMemcpyAsync(stg, rr, n * 8, cudaMemcpyHostToDevice, c->stream), "copy rho_r");
    LBCG_CUDA(cudaMemcpyAsync(stg + n, rb, n * 8, cudaMemcpyHostToDevice, c->stream), "copy rho_b");
    if (u) LBCG_CUDA(cudaMemcpyAsync(stg + 2 * n, u, n * 8 * c->D, cudaMemcpyHostToDevice, c->stream), "copy u");
    LBCG_CUDA(launch_init(c, stg, stg + n, u ? stg + 2 * n : nullptr, c->A), "init kernel");
    st = mirror_state(c);
    if (st) return st;
    LBCG_CUDA(cudaStreamSynchronize(c->stream), "init sync");
    c->fields = true;
    c->step = 0;
    return LBCG_OK;
}

static int drain_events(lbcg_ctx* c)
{
    for (size_t k = 0; k + 1 < c->ev_used; k += 2) {
        LBCG_CUDA(cudaEventSynchronize(c->ev_pool[k + 1]), "event sync");
        float ms = 0.f;
        LBCG_CUDA(cudaEventElapsedTime(&ms, c->ev_pool[k], c->ev_pool[k + 1]), "event elapsed");
        c->timed_ms += ms;
        c->timed_launches += 1;
    }
    c->ev_used = 0;
    return LBCG_OK;
}

static int next_events(lbcg_ctx* c, cudaEvent_t& e0, cudaEvent_t& e1)
{
    constexpr size_t kMaxPairs = 4096;
    if (c->ev_used + 2 > 2 * kMaxPairs) {
        int st = drain_events(c);
        if (st) return st;
    }
    while (c->ev_pool.size() < c->ev_used + 2) {
        cudaEvent_t e;
        LBCG_CUDA(cudaEventCreate(&e), "event create");
        c->ev_pool.push_back(e);
    }
    e0 = c->ev_pool[c->ev_used];
    e1 = c->ev_pool[c->ev_used + 1];
    c->ev_used += 2;
    return LBCG_OK;
}

static void drop_graphs(lbcg_ctx* c)
{
    for (int k = 0; k < 2; ++k) {
        if (c->graph[k]) cudaGraphExecDestroy(c->graph[k]);
        c->graph[k] = nullptr;
        c->graph_start[k] = nullptr;
    }
}

// port refill of A before a step, unless the step kernel that wrote A refilled the ghosts
static int refill_ports(lbcg_ctx* c)
{
    if (c->nghost > 0 && !(c->ghosts_fresh && step_fuses_ports(c)))
        LBCG_CUDA(launch_fill_ports(c, c->A), "port fill kernel");
    c->ghosts_fresh = true;
    return LBCG_OK;
}

// after a step kernel: its output buffer becomes A; its ghosts are refilled only if the
// kernel refills ports itself
static void finish_step(lbcg_ctx* c)
{
    std::swap(c->A, c->B);
    c->ghosts_fresh = step_fuses_ports(c);
}

// enqueue one step (port refill unless fused, fused kernel) on c->stream, swap the buffers
static int one_step(lbcg_ctx* c)
{
    const int st = refill_ports(c);
    if (st) return st;
    LBCG_CUDA(launch_step(c, c->A, c->B), "step kernel");
    finish_step(c);
    return LBCG_OK;
}

// graph of kGraphSteps steps starting from the current buffer A, captured on a private
// stream (capture is not allowed on the legacy default stream the caller may use)
static int graph_for_current(lbcg_ctx* c, cudaGraphExec_t& exec)
{
    const int k = c->A == c->graph_start[0] ? 0 : (c->A == c->graph_start[1] ? 1 : -1);
    if (k >= 0 && c->graph[k]) {
        exec = c->graph[k];
        return LBCG_OK;
    }
    const int slot = c->graph[0] ? 1 : 0;
    if (!c->cap_stream) LBCG_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking), "stream create");
    cudaStream_t user = c->stream;
    void* a0 = c->A;
    void* b0 = c->B;
    const bool fresh0 = c->ghosts_fresh;
    c->stream = c->cap_stream;
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    int st = LBCG_OK;
    if (e == cudaSuccess) {
        for (int t = 0; t < kGraphSteps && st == LBCG_OK; ++t) st = one_step(c);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
        if (st == LBCG_OK && e2 == cudaSuccess) {
            e = cudaGraphInstantiate(&c->graph[slot], g, 0);
        } else if (e2 != cudaSuccess) {
            e = e2;
        }
        if (g) cudaGraphDestroy(g);
    }
    c->stream = user;
    c->A = a0;
    c->B = b0;
    c->ghosts_fresh = fresh0;
    if (st) return st;
    if (e != cudaSuccess) return cuda_fail(e, "graph capture");
    c->graph_start[slot] = a0;
    exec = c->graph[slot];
    return LBCG_OK;
}

int lbcg_step(lbcg_ctx* c, long long nsteps)
{
    const lbcg::TraceRange trace("lbcg_step");
    int st = need(c, true);
    if (st) return st;
    if (nsteps < 0) return fail(LBCG_ERR_ARG, "negative step count");
    long long left = nsteps;
    if (left >= kGraphSteps) {
        // a graph of fused steps starts from refilled ghosts: refill once before it if needed
        if (step_fuses_ports(c) && !c->ghosts_fresh) {
            st = refill_ports(c);
            if (st) return st;
        }
        while (left >= kGraphSteps) {
            cudaGraphExec_t exec = nullptr;
            st = graph_for_current(c, exec);
            if (st) return st;
            LBCG_CUDA(cudaGraphLaunch(exec, c->stream), "graph launch");
            c->ghosts_fresh = step_fuses_ports(c);
            c->step += kGraphSteps;
            left -= kGraphSteps;
        }
    }
    for (; left > 0; --left) {
        if (c->timing) {
            st = refill_ports(c);
            if (st) return st;
            cudaEvent_t e0, e1;
            st = next_events(c, e0, e1);
            if (st) return st;
            LBCG_CUDA(cudaEventRecord(e0, c->stream), "event record");
            LBCG_CUDA(launch_step(c, c->A, c->B), "step kernel");
            LBCG_CUDA(cudaEventRecord(e1, c->stream), "event record");
            finish_step(c);
        } else {
            st = one_step(c);
            if (st) return st;
        }
        c->step += 1;
    }
    return LBCG_OK;
}

long long lbcg_step_count(const lbcg_ctx* c) { return c ? c->step : -1; }

// After a synchronisation: a step kernel whose shared-memory pipeline wait timed out left
// a nonzero status word (its results are invalid); report it once and clear it.
static int check_status(lbcg_ctx* c)
{
    if (!c->d_status) return LBCG_OK;
    int h = 0;
    LBCG_CUDA(cudaMemcpy(&h, c->d_status, sizeof(int), cudaMemcpyDeviceToHost), "status read");
    if (h == 0) return LBCG_OK;
    LBCG_CUDA(cudaMemset(c->d_status, 0, sizeof(int)), "status reset");
    if (h == kStatusBounds)
        return fail(LBCG_ERR_BOUNDS, "step kernel: an index outside its array (bounds-checked build); the state is invalid");
    return fail(LBCG_ERR_TIMEOUT, "step kernel: a bounded wait timed out; the state is invalid");
}

int lbcg_synchronize(lbcg_ctx* c)
{
    if (!c) return fail(LBCG_ERR_ARG, "null context");
    LBCG_CUDA(cudaStreamSynchronize(c->stream), "stream sync");
    return check_status(c);
}

int lbcg_get_fields_device(lbcg_ctx* c, double* rr, double* rb, double* u)
{
    int st = need(c, true);
    if (st) return st;
    if (!rr || !rb || !u) return fail(LBCG_ERR_ARG, "null output");
    LBCG_CUDA(launch_fields(c, c->A, rr, rb, u), "fields kernel");
    return LBCG_OK;
}

int lbcg_get_fields(lbcg_ctx* c, double* rr, double* rb, double* u)
{
    const lbcg::TraceRange trace("lbcg_get_fields");
    int st = need(c, true);
    if (st) return st;
    if (!rr || !rb || !u) return fail(LBCG_ERR_ARG, "null output");
    const size_t n = (size_t)c->n;
    void* sp = nullptr;
    st = scratch(c, n * 8 * (2 + c->D), &sp);
    if (st) return st;
    double* stg = (double*)sp;
    LBCG_CUDA(launch_fields(c, c->A, stg, stg + n, stg + 2 * n), "fields kernel");
    LBCG_CUDA(cudaMemcpyAsync(rr, stg, n * 8, cudaMemcpyDeviceToHost, c->stream), "copy rho_r");
    LBCG_CUDA(cudaMemcpyAsync(rb, stg + n, n * 8, cudaMemcpyDeviceToHost, c->stream), "copy rho_b");
    LBCG_CUDA(cudaMemcpyAsync(u, stg + 2 * n, n * 8 * c->D, cudaMemcpyDeviceToHost, c->stream), "copy u");
    LBCG_CUDA(cudaStreamSynchronize(c->stream), "fields sync");
    if (const int st_ = check_status(c)) return st_;
    return LBCG_OK;
}

int lbcg_get_populations(lbcg_ctx* c, double* f)
{
    int st = need(c, true);
    if (st) return st;
    if (!f) return fail(LBCG_ERR_ARG, "null output");
    const size_t n = (size_t)c->n;
    void* sp = nullptr;
    st = scratch(c, n * 8, &sp);
    if (st) return st;
    double* stg = (double*)sp;
    for (int k = 0; k < 2; ++k)
        for (int i = 0; i < c->Q; ++i) {
            LBCG_CUDA(launch_pop_plane_to_f64(c, c->A, k, i, stg), "population kernel");
            LBCG_CUDA(cudaMemcpyAsync(f + ((size_t)k * c->Q + i) * n, stg, n * 8, cudaMemcpyDeviceToHost,
                                      c->stream),
                      "copy populations");
            LBCG_CUDA(cudaStreamSynchronize(c->stream), "populations sync");
        }
    return check_status(c);
}

int lbcg_set_populations(lbcg_ctx* c, const double* f)
{
    int st = need(c, false);
    if (st) return st;
    if (!f) return fail(LBCG_ERR_ARG, "null input");
    const size_t n = (size_t)c->n;
    void* sp = nullptr;
    st = scratch(c, n * 16, &sp);
    if (st) return st;
    double* stg = (double*)sp;
    for (int i = 0; i < c->Q; ++i) {
        LBCG_CUDA(cudaMemcpyAsync(stg, f + (size_t)i * n, n * 8, cudaMemcpyHostToDevice, c->stream), "copy red");
        LBCG_CUDA(cudaMemcpyAsync(stg + n, f + ((size_t)c->Q + i) * n, n * 8, cudaMemcpyHostToDevice, c->stream),
                  "copy blue");
        LBCG_CUDA(launch_pops_from_f64(c, stg, c->A, i), "population kernel");
        LBCG_CUDA(cudaStreamSynchronize(c->stream), "populations sync");
    }
    st = mirror_state(c);
    if (st) return st;
    LBCG_CUDA(cudaStreamSynchronize(c->stream), "populations sync");
    c->fields = true;
    return LBCG_OK;
}

int lbcg_get_state(lbcg_ctx* c, void* host, size_t bytes)
{
    int st = need(c, true);
    if (st) return st;
    if (!host || bytes != c->state_bytes) return fail(LBCG_ERR_ARG, "host buffer must be lbcg_state_bytes long");
    LBCG_CUDA(cudaMemcpyAsync(host, c->A, bytes, cudaMemcpyDeviceToHost, c->stream), "copy state");
    LBCG_CUDA(cudaStreamSynchronize(c->stream), "state sync");
    if (const int st_ = check_status(c)) return st_;
    return LBCG_OK;
}

void* lbcg_current_state(lbcg_ctx* c) { return c && c->bound ? c->A : nullptr; }

int lbcg_set_state(lbcg_ctx* c, const void* host, size_t bytes)
{
    int st = need(c, false);
    if (st) return st;
    if (!host || bytes != c->state_bytes) return fail(LBCG_ERR_ARG, "host buffer must be lbcg_state_bytes long");
    LBCG_CUDA(cudaMemcpyAsync(c->A, host, bytes, cudaMemcpyHostToDevice, c->stream), "copy state");
    st = mirror_state(c);
    if (st) return st;
    LBCG_CUDA(cudaStreamSynchronize(c->stream), "state sync");
    if (const int st_ = check_status(c)) return st_;
    c->fields = true;
    return LBCG_OK;
}

// checkpoint file: "LBCGCKPT" | uint32 version 1 | lbcg_params | int64 step | uint64 bytes | state
int lbcg_save(lbcg_ctx* c, const char* path)
{
    int st = need(c, true);
    if (st) return st;
    if (!path) return fail(LBCG_ERR_ARG, "null path");
    std::vector<unsigned char> buf(c->state_bytes);
    st = lbcg_get_state(c, buf.data(), buf.size());
    if (st) return st;
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(LBCG_ERR_ARG, std::string("cannot open ") + path);
    const uint32_t ver = 1;
    const long long step = c->step;
    const uint64_t nb = c->state_bytes;
    bool ok = std::fwrite("LBCGCKPT", 1, 8, f) == 8 && std::fwrite(&ver, sizeof(ver), 1, f) == 1 &&
              std::fwrite(&c->p, sizeof(c->p), 1, f) == 1 && std::fwrite(&step, sizeof(step), 1, f) == 1 &&
              std::fwrite(&nb, sizeof(nb), 1, f) == 1 && std::fwrite(buf.data(), 1, buf.size(), f) == buf.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? LBCG_OK : fail(LBCG_ERR_ARG, std::string("write failed: ") + path);
}

int lbcg_load(lbcg_ctx* c, const char* path)
{
    int st = need(c, false);
    if (st) return st;
    if (!path) return fail(LBCG_ERR_ARG, "null path");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(LBCG_ERR_ARG, std::string("cannot open ") + path);
    char magic[8];
    uint32_t ver = 0;
    lbcg_params p;
    long long step = 0;
    uint64_t nb = 0;
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "LBCGCKPT", 8) == 0 &&
              std::fread(&ver, sizeof(ver), 1, f) == 1 && ver == 1 && std::fread(&p, sizeof(p), 1, f) == 1 &&
              std::fread(&step, sizeof(step), 1, f) == 1 && std::fread(&nb, sizeof(nb), 1, f) == 1;
    if (!ok) {
        std::fclose(f);
        return fail(LBCG_ERR_ARG, "not an lbcg checkpoint (version 1)");
    }
    if (p.lattice != c->p.lattice || p.nx != c->p.nx || p.ny != c->p.ny ||
        (c->p.lattice == LBCG_D3Q19 && p.nz != c->p.nz) || p.precision != c->p.precision || nb != c->state_bytes) {
        std::fclose(f);
        return fail(LBCG_ERR_ARG, "checkpoint lattice, box or precision differs from the context");
    }
    std::vector<unsigned char> buf(nb);
    ok = std::fread(buf.data(), 1, nb, f) == nb;
    std::fclose(f);
    if (!ok) return fail(LBCG_ERR_ARG, "truncated checkpoint");
    st = lbcg_set_state(c, buf.data(), buf.size());
    if (st) return st;
    c->step = step;
    return LBCG_OK;
}

int lbcg_observables(lbcg_ctx* c, const double centre[3], double r_in, double r_out, lbcg_obs* out)
{
    const lbcg::TraceRange trace("lbcg_observables");
    int st = need(c, true);
    if (st) return st;
    if (!centre || !out) return fail(LBCG_ERR_ARG, "null centre or output");
    LBCG_CUDA(launch_observables(c, c->A, centre, r_in, r_out, c->d_partials, c->d_result), "observable kernels");
    double res[2 * kObsSlots];
    LBCG_CUDA(cudaMemcpyAsync(res, c->d_result, sizeof(res), cudaMemcpyDeviceToHost, c->stream), "copy result");
    LBCG_CUDA(cudaStreamSynchronize(c->stream), "observables sync");
    if (const int st_ = check_status(c)) return st_;
    std::memset(out, 0, sizeof(*out));
    out->mass_r = res[0];
    out->mass_b = res[1];
    out->mom[0] = res[2];
    out->mom[1] = res[3];
    out->mom[2] = res[4];
    out->amount = res[5];
    out->umax = res[6];
    out->nonfinite = (int)res[7];
    out->r_eff = res[8];
    out->n_in = res[12];
    out->n_out = res[14];
    out->p_in = res[12] > 0 ? res[11] / res[12] : 0.0;
    out->p_out = res[14] > 0 ? res[13] / res[14] : 0.0;
    out->dp = out->p_in - out->p_out;
    out->step = c->step;
    if (out->nonfinite > 0) return fail(LBCG_ERR_DIVERGED, "non-finite or non-positive density at fluid sites");
    return LBCG_OK;
}

int lbcg_observables_noalloc(const lbcg_params* p, const void* dev_state, const uint8_t* dev_mask,
                             const double centre[3], double r_in, double r_out, void* stream, lbcg_obs* out)
{
    int st = validate(p);
    if (st) return st;
    if (!dev_state || !centre || !out) return fail(LBCG_ERR_ARG, "null state, centre or output");
    std::string err;
    st = noalloc_observables(p, dev_state, dev_mask, centre, r_in, r_out, stream, out, err);
    if (st) return fail(st, err);
    return LBCG_OK;
}

int lbcg_label(lbcg_ctx* c, int32_t* labels, int64_t* counts, double* volumes, int cap, int* n_drops)
{
    const lbcg::TraceRange trace("lbcg_label");
    int st = need(c, true);
    if (st) return st;
    if (!labels || !n_drops || cap < 0) return fail(LBCG_ERR_ARG, "null output");
    const size_t n = (size_t)c->n;
    // scratch: half[n] doubles | labels[n] ints | flag
    void* sp = nullptr;
    st = scratch(c, n * 12 + 16, &sp);
    if (st) return st;
    double* half = (double*)sp;
    int32_t* L = (int32_t*)(half + n);
    int* flag = (int*)(L + n + (n & 1));
    LBCG_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), c->stream), "clear flag");
    LBCG_CUDA(launch_label(c, c->A, L, half, flag), "label kernels");
    std::vector<double> h(n);
    int hflag = 0;
    LBCG_CUDA(cudaMemcpyAsync(labels, L, n * 4, cudaMemcpyDeviceToHost, c->stream), "copy labels");
    LBCG_CUDA(cudaMemcpyAsync(h.data(), half, n * 8, cudaMemcpyDeviceToHost, c->stream), "copy volumes");
    LBCG_CUDA(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "copy flag");
    LBCG_CUDA(cudaStreamSynchronize(c->stream), "label sync");
    if (const int st_ = check_status(c)) return st_;
    if (hflag) return fail(LBCG_ERR_TIMEOUT, "labelling iteration bound reached");
    // per-droplet count and volume in label order, sums in site order
    std::vector<int> slot(n, -1);
    int nd = 0;
    std::vector<int64_t> cnt;
    std::vector<double> vol;
    for (size_t s = 0; s < n; ++s) {
        const int lab = labels[s];
        if (lab < 0) continue;
        if (lab == (int)s) {
            slot[s] = nd++;
            cnt.push_back(0);
            vol.push_back(0.0);
        }
        const int k = slot[(size_t)lab];
        if (k < 0) return fail(LBCG_ERR_CUDA, "label points to a non-root site");
        cnt[k] += 1;
        vol[k] += h[s];
    }
    for (int k = 0; k < nd && k < cap; ++k) {
        if (counts) counts[k] = cnt[k];
        if (volumes) volumes[k] = vol[k];
    }
    *n_drops = nd;
    return LBCG_OK;
}

int lbcg_set_kernel_timing(lbcg_ctx* c, int enable)
{
    if (!c) return fail(LBCG_ERR_ARG, "null context");
    if (!enable && c->timing) {
        int st = drain_events(c);
        if (st) return st;
    }
    c->timing = enable != 0;
    c->timed_ms = 0.0;
    c->timed_launches = 0;
    return LBCG_OK;
}

int lbcg_kernel_time(lbcg_ctx* c, double* total_ms, long long* launches)
{
    if (!c || !total_ms || !launches) return fail(LBCG_ERR_ARG, "null argument");
    int st = drain_events(c);
    if (st) return st;
    *total_ms = c->timed_ms;
    *launches = c->timed_launches;
    c->timed_ms = 0.0;
    c->timed_launches = 0;
    return LBCG_OK;
}

int lbcg_get_launch(lbcg_ctx* c, int* rows, int* block_rows, int* variant)
{
    if (!c) return fail(LBCG_ERR_ARG, "null context");
    if (rows) *rows = c->kp.rows;
    if (block_rows) *block_rows = c->p.lattice == LBCG_D2Q9 ? 0 : c->block_rows;
    if (variant) *variant = effective_variant(c);
    return LBCG_OK;
}

int lbcg_get_grid(lbcg_ctx* c, long long* blocks, int* threads, int* kernels_per_step)
{
    if (!c) return fail(LBCG_ERR_ARG, "null context");
    const KParams& k = c->kp;
    long long b = 0;
    int t = 0;
    if (c->p.lattice == LBCG_D2Q9) {
        const long long warps = c->d_tiles ? (long long)k.ntiles : (long long)k.nsx * k.nsy;
        t = 256;
        b = (warps * 32 + t - 1) / t;
    } else {
        t = 32 * c->block_rows;
        b = c->d_tiles ? (long long)k.ntiles : (long long)k.nsx * k.nsy * k.nsz;
    }
    if (blocks) *blocks = b;
    if (threads) *threads = t;
    if (kernels_per_step) *kernels_per_step = 1 + (c->nghost > 0 && !step_fuses_ports(c) ? 1 : 0);
    return LBCG_OK;
}

int lbcg_set_launch(lbcg_ctx* c, int rows, int block_rows, int variant)
{
    if (!c) return fail(LBCG_ERR_ARG, "null context");
    // the moment march with shared-memory moments (variant 7, regularized collision) takes
    // blocks of up to 512 threads; every other kernel up to 256
    const int max_wy = variant == 7 && c->p.collision == LBCG_REG ? 16 : 8;
    if (rows < 0 || block_rows < 0 || (block_rows > 0 && (block_rows < 3 || block_rows > max_wy)) || variant < 0 ||
        variant > 9 || variant == 3 || variant == 4)
        return fail(LBCG_ERR_ARG,
                    "launch shape out of range (block_rows in 3..8, 3..16 with variant 7; variant in 0..2, 5..9)");
    c->rows = rows;
    c->block_rows = block_rows;
    c->variant = variant;
    fill_kparams(c);
    drop_graphs(c);
    return build_tiles(c);
}

}  // extern "C"
