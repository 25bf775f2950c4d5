// batch.cu -- many independent instances advanced together (lbcg_batch_*).
//
// A batch holds up to max_instances contexts of one lattice and storage precision.  Each
// lbcg_batch_step chunk replays one captured CUDA graph of graph_steps nodes; node k
// refills the port ghosts and runs the batched fused step for every instance with more
// than k steps left in the chunk.  Which instances take part, their buffers and step
// counts live in a device table the host rewrites before each replay, so admitting or
// retiring an instance never re-captures the graph (only a larger work list does).
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbcg_device.cuh"

using namespace lbcg;

namespace {
constexpr int kBatchGraphSteps = 32;   // default steps per captured graph
constexpr int kBatch2DRows = 16;       // default rows per D2Q9 warp strip
constexpr int kBatch3DRows = 8;        // default z-planes per D3Q19 tile
constexpr int kBatchStrips = 8;        // default D2Q9 strips (warps) per work item
}  // namespace

struct lbcg_batch {
    int lattice = 0, precision = 0, max_slots = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    std::vector<lbcg_ctx*> ctx;           // nullptr = free slot
    std::vector<long long> remaining;     // steps still to run
    std::vector<char> reported;           // completion already returned by poll
    std::vector<KParams> kp;              // per-slot launch-shaped parameters
    std::vector<std::vector<int>> tiles;  // per-slot D3Q19 fitted tiles (column, z-range), set at add
    BatchSlot* h_slots = nullptr;         // pinned, two tables (replays alternate between them)
    BatchSlot* d_slots = nullptr;
    std::vector<BatchItem> h_items, h_fill;
    BatchItem* d_items = nullptr;
    BatchItem* d_fill = nullptr;
    int* d_counts = nullptr;              // [0] step items, [1] fill items
    int items_cap = 0, fill_cap = 0;
    bool dirty = true;                    // membership changed: rebuild work lists
    cudaGraphExec_t graph = nullptr;
    cudaEvent_t done[2] = {nullptr, nullptr};  // last replay that read table 0 / 1
    long long nrep = 0;                   // replays launched
    lbcg_batch_shape shape{};             // launch shape after defaults (lbcg_batch_set_shape)
    int grid = 0;                         // persistent grid: SMs x resident blocks per SM
};

namespace {

thread_local std::string g_berr;

int bfail(int code, const std::string& m)
{
    g_berr = m;
    return code;
}

void drop_graph(lbcg_batch* b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
}

// rebuild the work lists of the occupied slots; grow device capacity if needed
int rebuild(lbcg_batch* b)
{
    b->h_items.clear();
    b->h_fill.clear();
    for (int s = 0; s < b->max_slots; ++s) {
        if (!b->ctx[s]) continue;
        const KParams& k = b->kp[s];
        if (b->lattice == LBCG_D2Q9) {
            const int strips = k.nsx * k.nsy, per = b->shape.strips_per_item;
            for (int f = 0; f < strips; f += per) b->h_items.push_back({s, f, std::min(per, strips - f), 0});
        } else {
            // the instance's block tiles that hold fluid, with fitted z-ranges (computed at add)
            const std::vector<int>& tiles = b->tiles[s];
            for (size_t t = 0; t + 1 < tiles.size(); t += 2)
                b->h_items.push_back({s, tiles[t] % k.nsx, tiles[t] / k.nsx, tiles[t + 1]});
        }
        const int ng = b->ctx[s]->nghost;
        for (int f = 0; f < ng; f += 64) b->h_fill.push_back({s, f, std::min(64, ng - f), 0});  // a thread per ghost
    }
    const int ni = (int)b->h_items.size(), nf = (int)b->h_fill.size();
    if (ni > b->items_cap || nf > b->fill_cap) {
        drop_graph(b);
        if (ni > b->items_cap) {
            cudaFree(b->d_items);
            b->items_cap = std::max(ni, 2 * b->items_cap);
            if (cudaMalloc(&b->d_items, sizeof(BatchItem) * b->items_cap) != cudaSuccess)
                return bfail(LBCG_ERR_NOMEM, "batch work list allocation failed");
        }
        if (nf > b->fill_cap) {
            cudaFree(b->d_fill);
            b->fill_cap = std::max(nf, std::max(64, 2 * b->fill_cap));
            if (cudaMalloc(&b->d_fill, sizeof(BatchItem) * b->fill_cap) != cudaSuccess)
                return bfail(LBCG_ERR_NOMEM, "batch refill list allocation failed");
        }
    }
    int counts[2] = {ni, nf};
    cudaError_t e = cudaSuccess;
    if (ni) e = cudaMemcpyAsync(b->d_items, b->h_items.data(), sizeof(BatchItem) * ni, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && nf)
        e = cudaMemcpyAsync(b->d_fill, b->h_fill.data(), sizeof(BatchItem) * nf, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_counts, counts, sizeof(counts), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(LBCG_ERR_CUDA, std::string("batch work lists: ") + cudaGetErrorString(e));
    b->dirty = false;
    return LBCG_OK;
}

int capture(lbcg_batch* b)
{
    if (b->graph) return LBCG_OK;
    if (!b->cap_stream && cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return bfail(LBCG_ERR_CUDA, "batch capture stream");
    cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bfail(LBCG_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(e));
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < b->shape.graph_steps && le == cudaSuccess; ++k) {
        le = launch_batch_fill(b->lattice, b->precision, b->d_slots, b->d_fill, b->d_counts + 1, b->fill_cap, k,
                               b->cap_stream);
        if (le == cudaSuccess)
            le = launch_batch_step(b->lattice, b->precision, b->d_slots, b->d_items, b->d_counts, k, b->grid,
                                   b->shape.block_rows, b->cap_stream);
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->cap_stream, &g);
    if (le != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bfail(LBCG_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(le != cudaSuccess ? le : e));
    }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(LBCG_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
    return LBCG_OK;
}

// shape after defaults; grid of the persistent kernel from the device's SM count
int apply_shape(lbcg_batch* b, const lbcg_batch_shape& in)
{
    lbcg_batch_shape sh = in;
    const bool d2 = b->lattice == LBCG_D2Q9;
    if (sh.rows <= 0) sh.rows = d2 ? kBatch2DRows : kBatch3DRows;
    sh.block_rows = d2 ? 0 : (sh.block_rows <= 0 ? 8 : sh.block_rows);
    sh.strips_per_item = d2 ? (sh.strips_per_item <= 0 ? kBatchStrips : sh.strips_per_item) : 0;
    if (sh.graph_steps <= 0) sh.graph_steps = kBatchGraphSteps;
    if (sh.rows > 65535 || (!d2 && (sh.block_rows < 3 || sh.block_rows > 8)) ||
        (d2 && (sh.strips_per_item < 1 || sh.strips_per_item > 8)) || sh.graph_steps < 2 || sh.graph_steps > 256 ||
        (sh.graph_steps & 1) || sh.blocks_per_sm < 0 || sh.blocks_per_sm > 32)
        return bfail(LBCG_ERR_ARG, "batch shape out of range (block_rows 3..8, strips_per_item 1..8, even "
                                   "graph_steps 2..256, blocks_per_sm 0..32)");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return bfail(LBCG_ERR_CUDA, "SM count query failed");
    const int fit = batch_resident_blocks(b->lattice, b->precision, d2 ? 8 : sh.block_rows);
    if (fit <= 0) return bfail(LBCG_ERR_CUDA, "occupancy query of the batched kernel failed");
    sh.blocks_per_sm = sh.blocks_per_sm <= 0 ? fit : std::min(sh.blocks_per_sm, fit);
    sh.sms = sms;
    b->shape = sh;
    b->grid = sms * sh.blocks_per_sm;
    return LBCG_OK;
}

// launch-shaped parameters and D3Q19 fitted tiles of slot s under the batch's shape
int shape_slot(lbcg_batch* b, int s)
{
    lbcg_ctx* c = b->ctx[s];
    b->kp[s] = make_kparams(c->p, c->dims, c->np, b->shape.rows, b->lattice == LBCG_D2Q9 ? 8 : b->shape.block_rows);
    b->tiles[s].clear();
    if (b->lattice != LBCG_D2Q9 && !fitted_tiles_3d(c, b->kp[s], b->shape.block_rows - 2, b->tiles[s]))
        return bfail(LBCG_ERR_CAPACITY, "instance with nz above 65535 in a batch");
    return LBCG_OK;
}

}  // namespace

extern "C" {

const char* lbcg_batch_last_error(void) { return g_berr.c_str(); }

int lbcg_batch_create(int lattice, int precision, int max_instances, void* stream, lbcg_batch** out)
{
    if (!out) return bfail(LBCG_ERR_ARG, "null output");
    *out = nullptr;
    if (lattice != LBCG_D2Q9 && lattice != LBCG_D3Q19) return bfail(LBCG_ERR_ARG, "unknown lattice");
    if (precision < LBCG_FP64 || precision > LBCG_FP16_SCALED) return bfail(LBCG_ERR_ARG, "unknown precision");
    if (max_instances < 1 || max_instances > 4096) return bfail(LBCG_ERR_ARG, "max_instances must be 1..4096");
    lbcg_batch* b = new (std::nothrow) lbcg_batch();
    if (!b) return bfail(LBCG_ERR_NOMEM, "host allocation failed");
    b->lattice = lattice;
    b->precision = precision;
    b->max_slots = max_instances;
    b->stream = (cudaStream_t)stream;
    cudaGetDevice(&b->device);
    b->ctx.assign(max_instances, nullptr);
    b->remaining.assign(max_instances, 0);
    b->reported.assign(max_instances, 0);
    b->kp.resize(max_instances);
    b->tiles.resize(max_instances);
    bool ok = cudaMallocHost(&b->h_slots, 2 * sizeof(BatchSlot) * max_instances) == cudaSuccess &&
              cudaMalloc(&b->d_slots, sizeof(BatchSlot) * max_instances) == cudaSuccess &&
              cudaMalloc(&b->d_counts, 2 * sizeof(int)) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->done[0], cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->done[1], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        lbcg_batch_destroy(b);
        return bfail(LBCG_ERR_NOMEM, "batch tables allocation failed");
    }
    std::memset(b->h_slots, 0, 2 * sizeof(BatchSlot) * max_instances);
    cudaMemsetAsync(b->d_slots, 0, sizeof(BatchSlot) * max_instances, b->stream);
    cudaMemsetAsync(b->d_counts, 0, 2 * sizeof(int), b->stream);
    const int st = apply_shape(b, lbcg_batch_shape{});
    if (st) {
        lbcg_batch_destroy(b);
        return st;
    }
    *out = b;
    return LBCG_OK;
}

int lbcg_batch_set_shape(lbcg_batch* b, const lbcg_batch_shape* shape)
{
    if (!b || !shape) return bfail(LBCG_ERR_ARG, "null argument");
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(LBCG_ERR_CUDA, cudaGetErrorString(e));
    const lbcg_batch_shape old = b->shape;
    int st = apply_shape(b, *shape);
    if (st) return st;
    for (int s = 0; s < b->max_slots; ++s) {
        if (!b->ctx[s]) continue;
        st = shape_slot(b, s);
        if (st) {
            b->shape = old;  // (the slot keeps its former parameters)
            return st;
        }
    }
    drop_graph(b);
    b->dirty = true;
    return LBCG_OK;
}

int lbcg_batch_get_shape(const lbcg_batch* b, lbcg_batch_shape* shape)
{
    if (!b || !shape) return bfail(LBCG_ERR_ARG, "null argument");
    *shape = b->shape;
    return LBCG_OK;
}

void lbcg_batch_destroy(lbcg_batch* b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    drop_graph(b);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (cudaEvent_t e : b->done)
        if (e) cudaEventDestroy(e);
    cudaFreeHost(b->h_slots);
    cudaFree(b->d_slots);
    cudaFree(b->d_items);
    cudaFree(b->d_fill);
    cudaFree(b->d_counts);
    delete b;
}

int lbcg_batch_add(lbcg_batch* b, lbcg_ctx* c, long long steps, int* slot)
{
    if (!b || !c || !slot) return bfail(LBCG_ERR_ARG, "null argument");
    if (steps < 0) return bfail(LBCG_ERR_ARG, "negative step count");
    if (c->p.lattice != b->lattice || c->p.precision != b->precision)
        return bfail(LBCG_ERR_ARG, "instance lattice/precision differs from the batch");
    if (!c->bound || !c->geometry || !c->fields) return bfail(LBCG_ERR_STATE, "instance not ready (state, geometry, fields)");
    if ((long long)2 * c->Q * (long long)c->np >= (1LL << 31) - 1)
        return bfail(LBCG_ERR_CAPACITY, "instance too large for the batched kernels (2Q planes >= 2^31 elements)");
    for (int s = 0; s < b->max_slots; ++s)
        if (b->ctx[s] == c) return bfail(LBCG_ERR_ARG, "instance already in the batch");
    int s = -1;
    for (int i = 0; i < b->max_slots; ++i)
        if (!b->ctx[i]) {
            s = i;
            break;
        }
    if (s < 0) return bfail(LBCG_ERR_CAPACITY, "batch is full");
    b->ctx[s] = c;
    b->remaining[s] = steps;
    b->reported[s] = 0;
    const int st = shape_slot(b, s);
    if (st) {
        b->ctx[s] = nullptr;
        b->remaining[s] = 0;
        return st;
    }
    b->dirty = true;
    *slot = s;
    return LBCG_OK;
}

int lbcg_batch_remove(lbcg_batch* b, int slot)
{
    if (!b || slot < 0 || slot >= b->max_slots || !b->ctx[slot]) return bfail(LBCG_ERR_ARG, "no such slot");
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(LBCG_ERR_CUDA, cudaGetErrorString(e));
    b->ctx[slot] = nullptr;
    b->remaining[slot] = 0;
    b->dirty = true;
    return LBCG_OK;
}

long long lbcg_batch_remaining(const lbcg_batch* b, int slot)
{
    if (!b || slot < 0 || slot >= b->max_slots || !b->ctx[slot]) return -1;
    return b->remaining[slot];
}

int lbcg_batch_step(lbcg_batch* b, long long max_steps)
{
    const TraceRange trace("lbcg_batch_step");
    if (!b) return bfail(LBCG_ERR_ARG, "null batch");
    if (max_steps < 0) return bfail(LBCG_ERR_ARG, "negative step count");
    long long done = 0;
    while (done < max_steps) {
        bool any = false;
        for (int s = 0; s < b->max_slots; ++s)
            if (b->ctx[s] && b->remaining[s] > 0) any = true;
        if (!any) break;
        if (b->dirty) {
            int st = rebuild(b);
            if (st) return st;
        }
        int st = capture(b);
        if (st) return st;
        // two pinned tables alternate between replays: the replay before the previous one
        // must have copied this table before it is rewritten (so the host runs ahead by a
        // replay instead of waiting for the GPU at every one)
        const int k = (int)(b->nrep & 1);
        BatchSlot* const tab = b->h_slots + (size_t)k * b->max_slots;
        cudaError_t e = cudaEventSynchronize(b->done[k]);
        if (e != cudaSuccess) return bfail(LBCG_ERR_CUDA, cudaGetErrorString(e));
        const long long chunk = std::min<long long>(b->shape.graph_steps, max_steps - done);
        for (int s = 0; s < b->max_slots; ++s) {
            BatchSlot& h = tab[s];
            lbcg_ctx* c = b->ctx[s];
            if (!c) {
                h.steps = 0;
                continue;
            }
            h.kp = b->kp[s];
            h.a = c->A;
            h.b = c->B;
            h.link = c->any_link ? c->d_link : nullptr;
            h.ghost = c->d_ghost;
            h.ghost_u = c->d_ghost_u;
            h.nghost = c->nghost;
            h.gpsi_a = gpsi_for(c, c->A);
            h.gpsi_b = gpsi_for(c, c->B);
            h.steps = (int)std::min<long long>(chunk, b->remaining[s]);
        }
        e = cudaMemcpyAsync(b->d_slots, tab, sizeof(BatchSlot) * b->max_slots, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaGraphLaunch(b->graph, b->stream);
        if (e == cudaSuccess) e = cudaEventRecord(b->done[k], b->stream);
        ++b->nrep;
        if (e != cudaSuccess) return bfail(LBCG_ERR_CUDA, std::string("batch replay: ") + cudaGetErrorString(e));
        for (int s = 0; s < b->max_slots; ++s) {
            lbcg_ctx* c = b->ctx[s];
            if (!c) continue;
            const int n = tab[s].steps;
            if (n & 1) std::swap(c->A, c->B);
            c->step += n;
            c->ghosts_fresh = false;  // the batched steps refill ports before each step only
            b->remaining[s] -= n;
        }
        done += chunk;
    }
    return LBCG_OK;
}

int lbcg_batch_poll(lbcg_batch* b, int* done_slots, int cap, int* ndone)
{
    if (!b || !ndone || (cap > 0 && !done_slots)) return bfail(LBCG_ERR_ARG, "null argument");
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(LBCG_ERR_CUDA, cudaGetErrorString(e));
    int n = 0;
    for (int s = 0; s < b->max_slots && n < cap; ++s)
        if (b->ctx[s] && b->remaining[s] == 0 && !b->reported[s]) {
            done_slots[n++] = s;
            b->reported[s] = 1;
        }
    *ndone = n;
    return LBCG_OK;
}

}  // extern "C"
