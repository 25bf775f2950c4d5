// lbcg_internal.h -- context structure, kernel parameter block and launcher
// declarations shared by the translation units of liblbcg.so.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/lbcg.h"
#include <nvtx3/nvToolsExt.h>

namespace lbcg {

// NVTX range around a host entry point (visible to Nsight tools; inert otherwise)
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

// Per-site link word: bits 0..Q-1 = "pull along direction i bounces back" (the
// upstream site x - c_i is a wall or outside a closed box face); bits 24..25 = site
// type (0 fluid, 1 wall, 2 port ghost).
constexpr uint32_t kTypeShift = 24;
constexpr uint32_t kTypeFluid = 0, kTypeWall = 1, kTypePort = 2;
// port sites: bits 0..23 of the link word hold the site's ghost-table row (when the context
// keeps a ghost-psi table; at most kGhostMask + 1 ghosts)
constexpr uint32_t kGhostMask = (1u << 24) - 1u;

// Physical constants in the arithmetic type of a kernel (float or double), so FP32
// kernels never touch FP64 arithmetic.
template <typename T>
struct Phys {
    T rho0;
    T half_inv_nu_r, half_inv_nu_b;   // 1/(2 nu_k), nu_k = (tau_k - 1/2)/3
    T A, beta, psi_wall;
    T phiR[3], phiB[3];               // phi_i^k per speed class (Eq. 7)
    T dphiR[3], dphiB[3];             // phi_i^k - w_i per speed class
    T wr0[3];                         // w_i rho0 per speed class
    T w[3], inv_w[3];                 // w_i and 1/w_i per speed class
    T scale_g, inv_scale_g;           // binary16 total-deviation scale
};

// Kernel parameter block, passed by value.
struct KParams {
    int nx, ny, nz;
    int per[3];
    size_t np;              // plane stride (elements)
    int collision;
    int lattice;
    int rows;               // marching length per warp / block
    int nsx, nsy, nsz;      // strips / blocks per axis
    int ntiles;             // entries of the active-tile list (0: launch every tile)
    int stall_test;         // failure-path test: TMA pipeline waits cannot complete (short limit)
    int* status;            // context status word (bounded-wait timeouts, bounds-checked build)
    Phys<float> pf;
    Phys<double> pd;
    double alpha_r, alpha_b;
};

template <typename T>
__host__ __device__ inline const Phys<T>& phys(const KParams& P);
template <>
__host__ __device__ inline const Phys<float>& phys<float>(const KParams& P) { return P.pf; }
template <>
__host__ __device__ inline const Phys<double>& phys<double>(const KParams& P) { return P.pd; }

// One instance of a batch as the batched kernels see it (device table, rewritten by the
// host before each graph launch; the captured graph itself never changes).
struct BatchSlot {
    KParams kp;              // launch shape: D2Q9 rows 16, D3Q19 8 x 8 blocks, 8 planes
    const void* a;           // current state (source of even steps of the launch)
    void* b;                 // other buffer
    const uint32_t* link;    // link words or nullptr
    const int* ghost;        // port ghost table or nullptr
    const double* ghost_u;
    int nghost;
    void* gpsi_a;            // ghost-psi tables (compute type) of buffers a and b, or nullptr
    void* gpsi_b;
    int steps;               // steps this launch advances the instance (0 = idle)
};
// work item: D2Q9 (slot, first strip, strip count <= 8, -); D3Q19 (slot, bx, by, z0 | z1 << 16)
// over the instance's fitted tiles;
// port refill (slot, first ghost, ghost count <= 64, -)
struct BatchItem {
    int slot, x, y, z;
};

KParams make_kparams(const lbcg_params& p, const int dims[3], size_t np, int rows, int block_rows);

constexpr int kMaxPartials = 1024;   // blocks of the deterministic reductions
constexpr int kObsSlots = 16;
constexpr int kGraphSteps = 32;   // steps per captured graph (even: A/B roles return)

}  // namespace lbcg

struct lbcg_ctx {
    lbcg_params p;
    int device = 0;
    cudaStream_t stream = nullptr;
    int Q = 9, D = 2;
    int dims[3] = {1, 1, 1};
    long long n = 0;        // sites
    size_t np = 0;          // padded plane length
    size_t state_bytes = 0;
    void* A = nullptr;      // current (post-collision) state
    void* B = nullptr;      // other buffer (scratch between steps)
    bool bound = false;
    bool geometry = false;
    bool fields = false;
    long long step = 0;

    // geometry tables (library-owned device memory)
    uint32_t* d_link = nullptr;
    bool any_link = false;             // any bounce bit or non-fluid site
    std::vector<uint8_t> mask;
    int nports = 0;
    lbcg_port ports[LBCG_MAX_PORTS];
    int nghost = 0;
    int* d_ghost = nullptr;            // [4][nghost]: site, inward neighbour, port, kind
    double* d_ghost_u = nullptr;       // [3][nghost] inlet velocity
    long long fluid_sites = 0;

    // tiles of the current launch shape that hold at least one fluid site (walled boxes only);
    // D3Q19 with ports: the ghost-table rows of each tile's x' sites, d_grow[d_gstart[t] ..
    // d_gstart[t+1]-1] for tile t (refilled by the moment marches after the tile)
    int* d_tiles = nullptr;
    int ntiles = 0;
    int* d_gstart = nullptr;
    int* d_grow = nullptr;
    std::vector<int> ghost_xp;         // inward neighbour x' of each ghost-table row (host copy)
    // the port ghosts of state A already hold the refill from A (written by a step kernel
    // that refills ports itself), so that kernel may run without a refill launch before it
    bool ghosts_fresh = false;
    // boxes with ports: psi of every ghost, one table of nghost values (compute type, 8-byte
    // slots) per state buffer; gpsi_buf[k] is the buffer table k belongs to.  Written by every
    // refill of that buffer's ghosts, read by the moment marches' port lanes
    double* d_gpsi = nullptr;
    const void* gpsi_buf[2] = {nullptr, nullptr};

    // read-back / labelling / staging scratch (allocated on first use, kept)
    void* d_scratch = nullptr;
    size_t scratch_bytes = 0;

    // reductions
    double* d_partials = nullptr;      // kMaxPartials * kObsSlots
    double* d_result = nullptr;        // 2 * kObsSlots

    // launch shape
    int rows = 0, block_rows = 0, variant = 0;

    // kernel timing: event pairs 2k, 2k+1 bracket the k-th timed launch since the last drain
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    double timed_ms = 0.0;
    long long timed_launches = 0;

    // CUDA graphs of kGraphSteps steps, one per starting buffer, captured on a private stream
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    void* graph_start[2] = {nullptr, nullptr};

    // TMA-staged step kernel: tensor maps of the two state buffers (CUtensorMap, 128 bytes,
    // encoded on first use for the buffer and block height they describe) and a device
    // status word its bounded pipeline waits set on timeout
    alignas(64) unsigned char tmap[2][128] = {};
    const void* tmap_buf[2] = {nullptr, nullptr};
    int tmap_wy[2] = {0, 0};
    int* d_status = nullptr;
    int stall_test = 0;  // LBCG_TEST_PIPELINE_STALL set when the context was created

    lbcg::KParams kp;
};

namespace lbcg {

// launchers (step.cu)
cudaError_t launch_step(lbcg_ctx* c, const void* a, void* b);
// the same for one storage format (step_kernels.cuh, one translation unit per format)
template <int PREC>
cudaError_t launch_step_prec(lbcg_ctx* c, const void* a, void* b);
template <int PREC>
int batch_resident_blocks_prec(int lattice, int wy);
template <int PREC>
cudaError_t launch_batch_step_prec(int lattice, const BatchSlot* slots, const BatchItem* items, const int* nitems,
                                   int k, int grid, int wy, cudaStream_t st);
// 32-bit element offsets suffice: all 2Q planes of the state below 2^31 elements
inline bool small_index(const lbcg_ctx* c) { return (long long)2 * c->Q * (long long)c->np < (1LL << 31) - 1; }
// cuTensorMapEncodeTiled from the driver (nullptr where unavailable), as a plain pointer (step.cu)
void* tma_encode_entry();
// ghost-psi table of state buffer `buf` (compute type), or nullptr without a table (api.cu)
void* gpsi_for(lbcg_ctx* c, const void* buf);
int effective_variant(const lbcg_ctx* c);  // the step kernel variant launch_step runs
bool tma_supported(const lbcg_ctx* c);     // the TMA-staged variant applies to this context
bool step_fuses_ports(const lbcg_ctx* c);  // the step kernel refills the port ghosts itself
// launchers (aux.cu)
cudaError_t launch_fill_ports(lbcg_ctx* c, void* a);
cudaError_t launch_init(lbcg_ctx* c, const double* rr, const double* rb, const double* u, void* a);
cudaError_t launch_fields(lbcg_ctx* c, const void* a, double* rr, double* rb, double* u);
cudaError_t launch_pop_plane_to_f64(lbcg_ctx* c, const void* a, int k, int i, double* out);
cudaError_t launch_pops_from_f64(lbcg_ctx* c, const double* f, void* a, int i);
cudaError_t launch_observables(lbcg_ctx* c, const void* a, const double centre[3], double r_in, double r_out,
                               double* d_partials, double* d_result);
cudaError_t launch_label(lbcg_ctx* c, const void* a, int32_t* parent, double* half, int* d_flag);
// batched launchers (step.cu, aux.cu): one graph node each
cudaError_t launch_batch_step(int lattice, int precision, const BatchSlot* slots, const BatchItem* items,
                              const int* nitems, int k, int grid, int wy, cudaStream_t st);
int batch_resident_blocks(int lattice, int precision, int wy);  // per SM, 0 if unknown
cudaError_t launch_batch_fill(int lattice, int precision, const BatchSlot* slots, const BatchItem* items,
                              const int* nitems, int cap, int k, cudaStream_t st);

void fill_kparams(lbcg_ctx* c);
int build_tiles(lbcg_ctx* c);
bool fitted_tiles_3d(const lbcg_ctx* c, const KParams& k, int ty, std::vector<int>& list);
// noalloc.cu
int noalloc_observables(const lbcg_params* p, const void* state, const uint8_t* mask, const double centre[3],
                        double r_in, double r_out, void* stream, lbcg_obs* out, std::string& err);
size_t storage_size(int precision);
// peak.cu
int fma_peak(int precision, void* stream, double* gflops, std::string& err);

}  // namespace lbcg
