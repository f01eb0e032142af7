// lbm_api_batch.cu -- the batch calls of the C ABI (include/lbm.h): many
// problems advanced by one persistent launch, its launch shape and
// autotuner, the neighbour lists that order its steps, and its test hooks.
#include "lbm_api_internal.h"
#include "lbm_batch_plan.h"

// ------------------------------------------------------------------ batch
struct lbm_batch {
    std::vector<lbm_ctx*> ctx;
    lbm_precision prec = LBM_FP32;
    cudaStream_t stream = nullptr;
    int device = 0;
    BatchProb* d_probs = nullptr;
    int4* d_tiles = nullptr;
    int ntiles = 0;
    std::vector<int4> tiles;           // host copy of the tile list
    std::vector<int> tiles_x, tiles_y, tile_base;   // per problem
    std::vector<char> periodic_x, periodic_y;       // per problem (any part of a side)
    // step ordering of the tile kernel: neighbour lists for grid nbr_grid
    int* d_nbr = nullptr;
    unsigned long long* d_done = nullptr;
    unsigned long long* d_epoch = nullptr;
    int nbr_cap = 0;    // CTAs the arrays hold
    int nbr_grid = -1;  // grid the lists were made for
    bool nbr_ok = false;
    long long* d_level = nullptr;
    unsigned* d_bar = nullptr;     // [0] arrivals, [1] generation
    unsigned* d_status = nullptr;
    unsigned* h_status = nullptr;
    long long step = 0;
    bool ready = false;
    int grid = 0;
    int npt = 1;                  // nodes per thread of the batch kernel (1 or 2)
    int max_grid[3] = {0, 0, 0};  // resident CTAs of a full wave, per npt
    int block = 0;                // steps per pass of the temporal-blocking kernel (0: tile kernel)
    bool tb_ok = false;           // every problem thin enough, none periodic in x
    int rows_max = 0;
    int4* d_segs = nullptr;
    int nsegs = 0;
    int tb_max_grid[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // per odd steps-per-pass 3, 5, 7
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_n = -1;
    int graph_state = 0;          // 1 captured and replayed, -1 capture failed
    cudaStream_t gstream = nullptr;  // private stream the graph runs on
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::string err;
};

namespace {
lbm_status bfail(lbm_batch* b, lbm_status s, const std::string& msg) {
    if (b) b->err = msg;
    else g_create_err = msg;
    return s;
}

// For each CTA of a grid, the other CTAs owning a tile next to one of its
// tiles in x or y, across periodic sides too.  False if some CTA has more
// than kBatchMaxNbr.
bool batch_neighbour_lists(const lbm_batch* b, int grid, std::vector<int>& out) {
    int tw = 0, th = 0;
    batch_tile_dims(&tw, &th);
    const int n = b->ntiles;
    std::vector<int> tp((size_t)n), tix((size_t)n), tiy((size_t)n);
    for (int t = 0; t < n; ++t) {
        tp[(size_t)t] = b->tiles[(size_t)t].x;
        tix[(size_t)t] = b->tiles[(size_t)t].y / tw;
        tiy[(size_t)t] = b->tiles[(size_t)t].z / th;
    }
    std::vector<unsigned char> px(b->periodic_x.begin(), b->periodic_x.end()),
        py(b->periodic_y.begin(), b->periodic_y.end());
    return batch_plan_neighbours(n, tp.data(), tix.data(), tiy.data(), b->tiles_x.data(), b->tiles_y.data(),
                                 b->tile_base.data(), px.data(), py.data(), grid,
                                 [&](int t) { return batch_tile_owner(t, n, grid); }, kBatchMaxNbr, out);
}

// Make the neighbour lists match the current grid (outside graph capture:
// waits for the stream, then copies synchronously).
cudaError_t batch_prepare_sync(lbm_batch* b) {
    if (b->block > 1 || b->nbr_grid == b->grid) return cudaSuccess;
    std::vector<int> lists;
    b->nbr_ok = b->grid <= b->nbr_cap && batch_neighbour_lists(b, b->grid, lists);
    b->nbr_grid = b->grid;
    if (!b->nbr_ok) return cudaSuccess;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_nbr, lists.data(), sizeof(int) * lists.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) b->nbr_ok = false;
    return e;
}

cudaError_t batch_launch(lbm_batch* b, int n) {
    auto go = [&](auto tm) {
        constexpr int TM = decltype(tm)::value;
        if (b->block > 1)
            return launch_batch_tb<TM>(b->d_probs, b->d_segs, b->nsegs, n, b->block, b->rows_max, b->d_level,
                                       b->d_bar, b->d_bar + 1, b->d_status, b->grid, b->stream);
        BatchSync sync;
        sync.nbr = b->nbr_ok && b->nbr_grid == b->grid ? b->d_nbr : nullptr;
        sync.done = b->d_done;
        sync.epoch = b->d_epoch;
        return launch_batch<TM>(b->d_probs, b->d_tiles, b->ntiles, n, b->d_level, b->d_bar, b->d_bar + 1,
                                b->d_status, sync, b->grid, b->npt, b->stream);
    };
    switch (b->prec) {
    case LBM_FP32_T64: return go(std::integral_constant<int, T_INT64>{});
    case LBM_FP32_TDF: return go(std::integral_constant<int, T_DF>{});
    case LBM_FP32_CONS: return go(std::integral_constant<int, T_CONS>{});
    default: return go(std::integral_constant<int, T_INT32>{});
    }
}
}  // namespace

extern "C" {

void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->gstream) cudaStreamDestroy(b->gstream);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    cudaFree(b->d_probs);
    cudaFree(b->d_tiles);
    cudaFree(b->d_nbr);
    cudaFree(b->d_done);
    cudaFree(b->d_epoch);
    cudaFree(b->d_segs);
    cudaFree(b->d_level);
    cudaFree(b->d_bar);
    cudaFree(b->d_status);
    cudaFreeHost(b->h_status);
    for (lbm_ctx* c : b->ctx) lbm_destroy(c);
    cudaGetLastError();
    delete b;
}

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err.c_str() : g_create_err.c_str(); }

lbm_status lbm_batch_create(int nprob, const lbm_problem* probs, lbm_precision prec, void* stream,
                            lbm_batch** out) {
    if (!out) return bfail(nullptr, LBM_E_INVAL, "out must not be NULL");
    *out = nullptr;
    if (nprob < 1 || !probs) return bfail(nullptr, LBM_E_INVAL, "lbm_batch_create: need nprob >= 1 problems");
    if (prec != LBM_FP32 && prec != LBM_FP32_T64 && prec != LBM_FP32_TDF && prec != LBM_FP32_CONS)
        return bfail(nullptr, LBM_E_INVAL, "lbm_batch_create: the batch runs the FP32 modes only");
    lbm_batch* b = new lbm_batch();
    b->prec = prec;
    b->stream = static_cast<cudaStream_t>(stream);
    cudaGetDevice(&b->device);
    for (int p = 0; p < nprob; ++p) {
        const lbm_problem& q = probs[p];
        lbm_ctx* c = nullptr;
        lbm_status s = lbm_create(q.nx, q.ny, q.b, q.tau, q.dt, q.dx, &q.dvm, &q.diss, q.bc, prec, stream, nullptr,
                                  nullptr, &c);
        if (s != LBM_OK) {
            std::string m = "problem " + std::to_string(p) + ": " + g_create_err;
            lbm_batch_destroy(b);
            return bfail(nullptr, s, m);
        }
        b->ctx.push_back(c);
    }
    int tw = 0, th = 0;
    batch_tile_dims(&tw, &th);
    std::vector<int4> tiles;
    for (int p = 0; p < nprob; ++p)
        for (int y0 = 0; y0 < probs[p].ny; y0 += th)
            for (int x0 = 0; x0 < probs[p].nx; x0 += tw) tiles.push_back(make_int4(p, x0, y0, 0));
    b->ntiles = (int)tiles.size();
    b->tiles = tiles;
    for (int p = 0, base = 0; p < nprob; ++p) {
        const int tx = (probs[p].nx + tw - 1) / tw, ty = (probs[p].ny + th - 1) / th;
        b->tiles_x.push_back(tx);
        b->tiles_y.push_back(ty);
        b->tile_base.push_back(base);
        base += tx * ty;
        auto periodic = [&](int side) {
            return probs[p].bc[side].kind_lo == LBM_BC_PERIODIC || probs[p].bc[side].kind_hi == LBM_BC_PERIODIC;
        };
        b->periodic_x.push_back(periodic(LBM_SIDE_LEFT) || periodic(LBM_SIDE_RIGHT));
        b->periodic_y.push_back(periodic(LBM_SIDE_BOTTOM) || periodic(LBM_SIDE_TOP));
    }
    // temporal blocking: thin problems without periodic x sides
    b->tb_ok = true;
    for (int p = 0; p < nprob && b->tb_ok; ++p) {
        b->rows_max = probs[p].ny > b->rows_max ? probs[p].ny : b->rows_max;
        if (probs[p].ny > kBatchTbRowsMax) b->tb_ok = false;
        for (int side = LBM_SIDE_LEFT; side <= LBM_SIDE_RIGHT; ++side)
            if (probs[p].bc[side].kind_lo == LBM_BC_PERIODIC || probs[p].bc[side].kind_hi == LBM_BC_PERIODIC)
                b->tb_ok = false;
    }
    std::vector<int4> segs;
    if (b->tb_ok) {
        const int sw = batch_tb_width();
        for (int p = 0; p < nprob; ++p)
            for (int x0 = 0; x0 < probs[p].nx; x0 += sw) segs.push_back(make_int4(p, x0, 0, 0));
    }
    b->nsegs = (int)segs.size();
    std::vector<BatchProb> hp(nprob);
    int bbx = 0, bby = 0;
    batch_box_dims(&bbx, &bby);
    for (int p = 0; p < nprob; ++p) {
        hp[p].f[0] = static_cast<float*>(b->ctx[p]->f[0]);
        hp[p].f[1] = static_cast<float*>(b->ctx[p]->f[1]);
        hp[p].M = b->ctx[p]->mf;
        hp[p].G = b->ctx[p]->gf;
        // a problem that wraps in y inside its tile needs only its interior rows
        hp[p].wrap = batch_wraps_in_tile(hp[p].G) ? 1 : 0;
        const int rows = hp[p].wrap ? th : bby;
        hp[p].box_bytes = (unsigned)(sizeof(float) * 9 * bbx * rows);
        for (int k = 0; k < 2; ++k)
            if (!make_tmap_box(&hp[p].tm[k], b->ctx[p]->f[k], *b->ctx[p], bbx, rows)) {
                lbm_batch_destroy(b);
                return bfail(nullptr, LBM_E_CUDA, "lbm_batch_create: tensor maps unavailable on this driver");
            }
    }
    // each tile entry carries what issuing its copy needs from its problem:
    // the box's bytes, and (top bit) whether the box starts one row lower
    for (int4& t : tiles) t.w = (int)(hp[(size_t)t.x].box_bytes | (hp[(size_t)t.x].wrap ? 0x80000000u : 0u));
    b->tiles = tiles;
    cudaError_t e = dev_malloc((void**)&b->d_probs, sizeof(BatchProb) * nprob);
    if (e == cudaSuccess) e = dev_malloc((void**)&b->d_tiles, sizeof(int4) * tiles.size());
    if (e == cudaSuccess && b->tb_ok) e = dev_malloc((void**)&b->d_segs, sizeof(int4) * segs.size());
    if (e == cudaSuccess) e = dev_malloc((void**)&b->d_level, sizeof(long long));
    if (e == cudaSuccess) e = dev_malloc((void**)&b->d_bar, 2 * sizeof(unsigned));
    if (e == cudaSuccess) e = dev_malloc((void**)&b->d_status, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_status, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->gstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_probs, hp.data(), sizeof(BatchProb) * nprob, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_tiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess && b->tb_ok)
        e = cudaMemcpyAsync(b->d_segs, segs.data(), sizeof(int4) * segs.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_bar, 0, 2 * sizeof(unsigned), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_status, 0, sizeof(unsigned), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_level, 0, sizeof(long long), b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        std::string m = std::string("lbm_batch_create: ") + cudaGetErrorString(e);
        lbm_batch_destroy(b);
        return bfail(nullptr, e == cudaErrorMemoryAllocation ? LBM_E_NOMEM : LBM_E_CUDA, m);
    }
    for (int npt = 1; npt <= 2; ++npt)
        b->max_grid[npt] = prec == LBM_FP32_T64    ? batch_max_grid<T_INT64>(npt)
                           : prec == LBM_FP32_TDF  ? batch_max_grid<T_DF>(npt)
                           : prec == LBM_FP32_CONS ? batch_max_grid<T_CONS>(npt)
                                                   : batch_max_grid<T_INT32>(npt);
    b->nbr_cap = b->max_grid[1] > b->max_grid[2] ? b->max_grid[1] : b->max_grid[2];
    e = dev_malloc((void**)&b->d_nbr, sizeof(int) * (size_t)b->nbr_cap * kBatchMaxNbr);
    // one counter per CTA, and one more (index nbr_cap) that no CTA ever
    // publishes to (lbm_batch_plant_stall)
    if (e == cudaSuccess) e = dev_malloc((void**)&b->d_done, sizeof(unsigned long long) * (size_t)(b->nbr_cap + 1));
    if (e == cudaSuccess) e = dev_malloc((void**)&b->d_epoch, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(b->d_done, 0, sizeof(unsigned long long) * (size_t)(b->nbr_cap + 1));
    if (e == cudaSuccess) e = cudaMemset(b->d_epoch, 0, sizeof(unsigned long long));
    if (e != cudaSuccess) {
        std::string m = std::string("lbm_batch_create: ") + cudaGetErrorString(e);
        lbm_batch_destroy(b);
        return bfail(nullptr, e == cudaErrorMemoryAllocation ? LBM_E_NOMEM : LBM_E_CUDA, m);
    }
    b->npt = 1;
    b->grid = b->max_grid[1] < b->ntiles ? b->max_grid[1] : b->ntiles;
    if (b->tb_ok)
        for (int ns = 3; ns <= 7; ns += 2)
            b->tb_max_grid[ns] = prec == LBM_FP32_T64    ? batch_tb_max_grid<T_INT64>(ns, b->rows_max)
                                 : prec == LBM_FP32_TDF  ? batch_tb_max_grid<T_DF>(ns, b->rows_max)
                                 : prec == LBM_FP32_CONS ? batch_tb_max_grid<T_CONS>(ns, b->rows_max)
                                                         : batch_tb_max_grid<T_INT32>(ns, b->rows_max);
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_init(lbm_batch* b, const void* const* rho, const void* const* ux, const void* const* uy,
                          const void* const* T) {
    if (!b || !rho || !ux || !uy || !T) return bfail(b, LBM_E_INVAL, "lbm_batch_init: NULL argument");
    for (size_t p = 0; p < b->ctx.size(); ++p) {
        lbm_status s = lbm_init(b->ctx[p], rho[p], ux[p], uy[p], T[p]);
        if (s != LBM_OK) return bfail(b, s, "problem " + std::to_string(p) + ": " + b->ctx[p]->err);
    }
    cudaSetDevice(b->device);
    // the step counters and the grid barrier's words too: a launch that gave
    // up may have left the counters ahead of the epoch and the barrier with
    // arrivals that never completed
    if (cudaMemsetAsync(b->d_level, 0, sizeof(long long), b->stream) != cudaSuccess ||
        cudaMemsetAsync(b->d_status, 0, sizeof(unsigned), b->stream) != cudaSuccess ||
        cudaMemsetAsync(b->d_bar, 0, 2 * sizeof(unsigned), b->stream) != cudaSuccess ||
        cudaMemsetAsync(b->d_done, 0, sizeof(unsigned long long) * (size_t)(b->nbr_cap + 1), b->stream) !=
            cudaSuccess ||
        cudaMemsetAsync(b->d_epoch, 0, sizeof(unsigned long long), b->stream) != cudaSuccess)
        return bfail(b, LBM_E_CUDA, "lbm_batch_init: clearing the batch state failed");
    b->step = 0;
    b->ready = true;
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int n) {
    NvtxRange nvtx_range("lbm_batch_step");
    if (!b) return bfail(nullptr, LBM_E_INVAL, "NULL batch");
    if (n < 0) return bfail(b, LBM_E_INVAL, "lbm_batch_step: n must be >= 0");
    if (!b->ready) return bfail(b, LBM_E_STATE, "lbm_batch_step before lbm_batch_init");
    if (n == 0) return LBM_OK;
    cudaSetDevice(b->device);
    cudaError_t e = batch_prepare_sync(b);
    if (e != cudaSuccess) return bfail(b, LBM_E_CUDA, std::string("lbm_batch_step: ") + cudaGetErrorString(e));
    // One graph (a single cooperative kernel node) per step count, captured on
    // a private stream and replayed there, ordered after and before the
    // caller's stream by events; replays read the level from device memory,
    // so one graph serves every call with the same n.
    if (b->graph_state >= 0 && b->graph_n != n) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
        b->graph_n = -1;
        cudaStream_t keep = b->stream;
        b->stream = b->gstream;  // batch_launch queues on b->stream
        cudaGraph_t g = nullptr;
        cudaError_t be = cudaStreamBeginCapture(b->gstream, cudaStreamCaptureModeThreadLocal);
        cudaError_t le = be == cudaSuccess ? batch_launch(b, n) : be;
        cudaError_t ce = be == cudaSuccess ? cudaStreamEndCapture(b->gstream, &g) : be;
        cudaError_t ie = (le == cudaSuccess && ce == cudaSuccess && g) ? cudaGraphInstantiate(&b->exec, g, 0) : le;
        b->stream = keep;
        if (le == cudaSuccess && ce == cudaSuccess && ie == cudaSuccess && g) {
            b->graph = g;
            b->graph_n = n;
            b->graph_state = 1;
        } else {
            if (g) cudaGraphDestroy(g);
            b->exec = nullptr;
            b->graph_state = -1;
            b->err = std::string("graph capture of the batch launch failed (") +
                     cudaGetErrorString(le != cudaSuccess ? le : (ce != cudaSuccess ? ce : ie)) +
                     "); launching directly";
        }
        cudaGetLastError();
    }
    if (b->exec && b->graph_n == n) {
        e = cudaEventRecord(b->ev_in, b->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->gstream, b->ev_in, 0);
        if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->gstream);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_out, b->gstream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_out, 0);
    } else {
        e = batch_launch(b, n);
    }
    if (e != cudaSuccess) return bfail(b, LBM_E_CUDA, std::string("lbm_batch_step: ") + cudaGetErrorString(e));
    b->step += n;
    for (lbm_ctx* c : b->ctx) {
        c->step = b->step;
        c->cur = (int)(b->step & 1);
    }
    return LBM_OK;
}

lbm_status lbm_batch_sync(lbm_batch* b) {
    if (!b) return bfail(nullptr, LBM_E_INVAL, "NULL batch");
    cudaSetDevice(b->device);
    if (cudaMemcpyAsync(b->h_status, b->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return bfail(b, LBM_E_CUDA, "lbm_batch_sync: synchronising failed");
    if (*b->h_status & ST_TIMEOUT) return bfail(b, LBM_E_TIMEOUT, "a bounded wait between the batch kernel's CTAs gave up");
    if (*b->h_status & ST_NONPHYSICAL) return bfail(b, LBM_E_NONPHYSICAL, "a problem went non-physical");
    return LBM_OK;
}

lbm_ctx* lbm_batch_problem(lbm_batch* b, int p) {
    if (!b || p < 0 || p >= (int)b->ctx.size()) return nullptr;
    return b->ctx[(size_t)p];
}

lbm_status lbm_batch_info(const lbm_batch* b, int* grid, int* ntiles, int* graph) {
    if (!b) return LBM_E_INVAL;
    if (grid) *grid = b->grid;
    if (ntiles) *ntiles = b->ntiles;
    if (graph) *graph = b->graph_state;
    return LBM_OK;
}

}  // extern "C"

// ------------------------------------------------------- batch launch shape
namespace {
void batch_drop_graph(lbm_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->graph_n = -1;
    if (b->graph_state > 0) b->graph_state = 0;
}
}  // namespace

extern "C" {

lbm_status lbm_batch_set_launch(lbm_batch* b, const lbm_batch_launch* l) {
    if (!b || !l) return bfail(b, LBM_E_INVAL, "lbm_batch_set_launch: NULL argument");
    int full = 0;
    if (l->block > 1) {
        if (l->block != 3 && l->block != 5 && l->block != 7)
            return bfail(b, LBM_E_INVAL, "lbm_batch_set_launch: block must be 0, 1, 3, 5 or 7");
        if (!b->tb_ok)
            return bfail(b, LBM_E_INVAL,
                         "lbm_batch_set_launch: temporal blocking needs problems of at most " +
                             std::to_string(kBatchTbRowsMax) + " rows and no periodic x sides");
        full = b->tb_max_grid[l->block] < b->nsegs ? b->tb_max_grid[l->block] : b->nsegs;
        if (full < 1) return bfail(b, LBM_E_INVAL, "lbm_batch_set_launch: the blocking kernel does not fit");
    } else {
        if (l->block < 0) return bfail(b, LBM_E_INVAL, "lbm_batch_set_launch: block must be 0, 1, 3, 5 or 7");
        if (l->npt != 1 && l->npt != 2) return bfail(b, LBM_E_INVAL, "lbm_batch_set_launch: npt must be 1 or 2");
        full = b->max_grid[l->npt] < b->ntiles ? b->max_grid[l->npt] : b->ntiles;
    }
    if (l->grid < 0 || l->grid > full)
        return bfail(b, LBM_E_INVAL, "lbm_batch_set_launch: grid must lie in [0, " + std::to_string(full) + "]");
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    b->block = l->block > 1 ? l->block : 0;
    b->npt = l->block > 1 ? 1 : l->npt;
    b->grid = l->grid == 0 ? full : l->grid;
    batch_drop_graph(b);
    return LBM_OK;
}

lbm_status lbm_batch_set_wait_limit(double seconds) {
    if (!(seconds > 0.0) || seconds > 60.0) return LBM_E_INVAL;
    int dev = 0, khz = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess ||
        khz <= 0) {
        cudaGetLastError();
        return LBM_E_CUDA;
    }
    const long long cycles = (long long)(seconds * (double)khz * 1e3);
    if (batch_set_wait_cycles(cycles < 1 ? 1 : cycles) != cudaSuccess) {
        cudaGetLastError();
        return LBM_E_CUDA;
    }
    return LBM_OK;
}

lbm_status lbm_batch_plant_stall(lbm_batch* b, int cta) {
    if (!b) return bfail(nullptr, LBM_E_INVAL, "NULL batch");
    cudaSetDevice(b->device);
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess) e = batch_prepare_sync(b);
    if (e != cudaSuccess) return bfail(b, LBM_E_CUDA, std::string("lbm_batch_plant_stall: ") + cudaGetErrorString(e));
    if (cta < 0) {  // back to the lists of the current grid
        b->nbr_grid = -1;
        e = batch_prepare_sync(b);
        batch_drop_graph(b);
        return e == cudaSuccess ? LBM_OK : bfail(b, LBM_E_CUDA, "lbm_batch_plant_stall: restoring the lists failed");
    }
    if (b->block > 1 || !b->nbr_ok)
        return bfail(b, LBM_E_STATE, "lbm_batch_plant_stall: the current launch shape has no neighbour lists");
    if (cta >= b->grid)
        return bfail(b, LBM_E_INVAL, "lbm_batch_plant_stall: cta must lie in [0, " + std::to_string(b->grid) + ")");
    std::vector<int> lists;
    batch_neighbour_lists(b, b->grid, lists);
    int* row = lists.data() + (size_t)cta * kBatchMaxNbr;
    int j = 0;
    while (j < kBatchMaxNbr - 1 && row[j] >= 0) ++j;
    row[j] = b->nbr_cap;  // a counter no CTA publishes to
    e = cudaMemcpy(b->d_nbr, lists.data(), sizeof(int) * lists.size(), cudaMemcpyHostToDevice);
    batch_drop_graph(b);
    return e == cudaSuccess ? LBM_OK : bfail(b, LBM_E_CUDA, "lbm_batch_plant_stall: copying the lists failed");
}

lbm_status lbm_batch_get_launch(const lbm_batch* b, lbm_batch_launch* l) {
    if (!b || !l) return LBM_E_INVAL;
    l->npt = b->npt;
    l->grid = b->grid;
    l->block = b->block;
    return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch* b, int steps, lbm_batch_launch* best, double* ms, int* n_candidates) {
    NvtxRange nvtx_range("lbm_batch_autotune");
    if (!b) return bfail(nullptr, LBM_E_INVAL, "NULL batch");
    if (steps < 1) return bfail(b, LBM_E_INVAL, "lbm_batch_autotune: steps must be >= 1");
    if (!b->ready) return bfail(b, LBM_E_STATE, "lbm_batch_autotune before lbm_batch_init");
    cudaSetDevice(b->device);
    // candidates: nodes per thread 1 or 2, a full wave or half of one
    lbm_batch_launch cand[8];
    int nc = 0;
    for (int npt = 1; npt <= 2; ++npt) {
        const int full = b->max_grid[npt] < b->ntiles ? b->max_grid[npt] : b->ntiles;
        cand[nc++] = {npt, full, 0};
        if (full >= 2) cand[nc++] = {npt, full / 2, 0};
    }
    if (b->tb_ok)
        for (int ns = 3; ns <= 7; ns += 2) {
            const int full = b->tb_max_grid[ns] < b->nsegs ? b->tb_max_grid[ns] : b->nsegs;
            if (full >= 1) cand[nc++] = {1, full, ns};
        }
    // save every problem's current level, the level counter and the status
    const int cur = (int)(b->step & 1);
    size_t total = 0;
    for (lbm_ctx* c : b->ctx) total += level_bytes(c);
    unsigned char* save = nullptr;
    long long* d_lsave = nullptr;
    unsigned* d_ssave = nullptr;
    cudaError_t e = dev_malloc((void**)&save, total);
    if (e == cudaSuccess) e = dev_malloc((void**)&d_lsave, sizeof(long long));
    if (e == cudaSuccess) e = dev_malloc((void**)&d_ssave, sizeof(unsigned));
    size_t off = 0;
    for (lbm_ctx* c : b->ctx) {
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(save + off, c->f[cur], level_bytes(c), cudaMemcpyDeviceToDevice, b->stream);
        off += level_bytes(c);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_lsave, b->d_level, sizeof(long long), cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_ssave, b->d_status, sizeof(unsigned), cudaMemcpyDeviceToDevice, b->stream);
    auto restore = [&]() {
        cudaError_t r = cudaSuccess;
        size_t o = 0;
        for (lbm_ctx* c : b->ctx) {
            if (r == cudaSuccess)
                r = cudaMemcpyAsync(c->f[cur], save + o, level_bytes(c), cudaMemcpyDeviceToDevice, b->stream);
            o += level_bytes(c);
        }
        if (r == cudaSuccess)
            r = cudaMemcpyAsync(b->d_level, d_lsave, sizeof(long long), cudaMemcpyDeviceToDevice, b->stream);
        if (r == cudaSuccess)
            r = cudaMemcpyAsync(b->d_status, d_ssave, sizeof(unsigned), cudaMemcpyDeviceToDevice, b->stream);
        return r;
    };
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    const int keep_npt = b->npt, keep_grid = b->grid, keep_block = b->block;
    int bi = -1;
    float bms = 0.0f;
    for (int k = 0; k < nc && e == cudaSuccess; ++k) {
        b->npt = cand[k].npt;
        b->grid = cand[k].grid;
        b->block = cand[k].block;
        e = batch_prepare_sync(b);
        if (e == cudaSuccess) e = batch_launch(b, 1);  // untimed: first launch of the variant
        if (e == cudaSuccess) e = restore();
        if (e == cudaSuccess) e = cudaEventRecord(t0, b->stream);
        if (e == cudaSuccess) e = batch_launch(b, steps);
        if (e == cudaSuccess) e = cudaEventRecord(t1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        float m = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&m, t0, t1);
        if (e == cudaSuccess) e = restore();
        if (e == cudaSuccess && ms) ms[k] = m / steps;
        if (e == cudaSuccess && (bi < 0 || m < bms)) {
            bi = k;
            bms = m;
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    cudaFree(save);
    cudaFree(d_lsave);
    cudaFree(d_ssave);
    if (e != cudaSuccess || bi < 0) {
        b->npt = keep_npt;
        b->grid = keep_grid;
        b->block = keep_block;
        return bfail(b, LBM_E_CUDA, std::string("lbm_batch_autotune: ") + cudaGetErrorString(e));
    }
    b->npt = cand[bi].npt;
    b->grid = cand[bi].grid;
    b->block = cand[bi].block;
    batch_drop_graph(b);
    if (best) *best = cand[bi];
    if (n_candidates) *n_candidates = nc;
    return LBM_OK;
}

}  // extern "C"
