// pog_solve_noalloc: the whole solve (what pog_build + pog_maxflow + pog_surface do)
// for callers that must not allocate, with every scratch word in one file-scope device
// array instead of memory from cudaMalloc. See include/pog.h for the contract.
#include <cstddef>
#include <cstring>

#include "pog.h"
#include "pog_internal.cuh"
#include "pog_launch.h"

namespace {

// The scratch array. In host code its name is only a stand-in for the device object:
// its device address comes from cudaGetSymbolAddress (on every call, below).
static __device__ __align__(256) unsigned char g_noalloc_scratch[POG_NOALLOC_SCRATCH_BYTES];

constexpr int kGapLevels = 1 << 20;        // labels tracked by the gap bitmap
constexpr int kSweepsPerRelabel = 64;      // fixed: this path keeps no timing events
constexpr int kTileSweeps = 8;
constexpr int kNodeOps = 4;
constexpr int kMaxRounds = 1 << 20;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

pog_status from_cuda(cudaError_t e) { return e == cudaSuccess ? POG_OK : POG_E_CUDA; }

#define NA_TRY_CUDA(expr)                                \
    do {                                                 \
        const pog_status _s = from_cuda((expr));         \
        if (_s != POG_OK) return _s;                     \
    } while (0)
#define NA_TRY(expr)                                     \
    do {                                                 \
        const pog_status _s = (expr);                    \
        if (_s != POG_OK) return _s;                     \
    } while (0)

// Device address of the scratch array in the current device's context. Looked up on every
// call, so a context created anew (after cudaDeviceReset) is never given a stale address;
// once the module is loaded in a context the lookup allocates nothing.
pog_status scratch_address(void **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return POG_E_CUDA;
    *out = p;
    return POG_OK;
}

struct Carve {
    char *p;
    size_t used;
    template <class T>
    T *take(size_t bytes) {
        T *r = reinterpret_cast<T *>(p + used);
        used += align_up(bytes, 256);
        return r;
    }
};

// Bytes of scratch a volume needs (the same words as the allocating path, minus the
// heights, which go straight to the caller's buffer, and the relabel trace).
size_t scratch_bytes(int X, int Y, int Z, int alpha) {
    const size_t N = (size_t)X * Y * Z;
    const int arrays = alpha > 0 ? 10 : 8;
    pog::Grid dims{};
    dims.X = X;
    dims.Y = Y;
    dims.Z = Z;
    const size_t tiles = (size_t)pog::tile_count_max(dims);
    return (arrays + 2) * align_up(N * 4, 256) + align_up((N + 31) / 32 * 4, 256) + align_up(4 * tiles * 4, 256) + 256 +
           align_up(sizeof(pog::BfsSync), 256) + 2 * align_up(sizeof(pog::DevCounters), 256) + kGapLevels / 8 +
           align_up(sizeof(pog::Grid), 256) + 2 * 256;
}

// The union counters (`host[0]`) and the volume's counters (`host[1]`) to host memory.
pog_status read_counters(const pog::DevCounters *uctr, const pog::DevCounters *vctr, pog::DevCounters *host,
                         cudaStream_t st) {
    NA_TRY_CUDA(cudaMemcpyAsync(host, uctr, sizeof(*host), cudaMemcpyDeviceToHost, st));
    NA_TRY_CUDA(cudaMemcpyAsync(host + 1, vctr, sizeof(*host), cudaMemcpyDeviceToHost, st));
    NA_TRY_CUDA(cudaStreamSynchronize(st));
    const int err = host[0].error | host[1].error;
    if (err & POG_ERR_TIMEOUT) return POG_E_TIMEOUT;
    if (err) return POG_E_OVERFLOW;
    return POG_OK;
}

}  // namespace

extern "C" pog_status pog_solve_noalloc(const int32_t *cost_dev, int32_t X, int32_t Y, int32_t Z, int32_t delta,
                                        int32_t alpha, const pog_options *opt, void *stream, int64_t *flow_out,
                                        int32_t *heights_dev) {
    if (!cost_dev || !flow_out || !heights_dev || X < 1 || Y < 1 || Z < 1 || delta < 0 || alpha < 0 ||
        alpha >= (1 << 30))
        return POG_E_INVALID;
    if ((long long)X * Y * Z >= (1ll << 31) - 64) return POG_E_INVALID;
    if (scratch_bytes(X, Y, Z, alpha) > (size_t)POG_NOALLOC_SCRATCH_BYTES) return POG_E_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void *base = nullptr;
    NA_TRY(scratch_address(&base));

    const int sweeps = (opt && opt->sweeps_per_relabel > 0) ? opt->sweeps_per_relabel : kSweepsPerRelabel;
    const int tile_sweeps = (opt && opt->tile_sweeps > 0) ? opt->tile_sweeps : kTileSweeps;
    const int max_rounds = (opt && opt->max_rounds > 0) ? opt->max_rounds : kMaxRounds;
    const int flags = opt ? opt->flags : 0;
    const int bfs_blocks = (opt && opt->bfs_blocks_per_sm > 0) ? opt->bfs_blocks_per_sm : 0;

    const size_t N = (size_t)X * Y * Z;
    pog::Grid g{};
    g.X = X;
    g.Y = Y;
    g.Z = Z;
    g.delta = delta;
    g.alpha = alpha;
    g.N = (int)N;
    Carve c{static_cast<char *>(base), 0};
    g.lab = c.take<int32_t>(N * 4);
    g.exc = c.take<int32_t>(N * 4);
    g.snk = c.take<int32_t>(N * 4);
    g.fdn = c.take<int32_t>(N * 4);
    for (auto &f : g.fh) f = c.take<int32_t>(N * 4);
    for (auto &s : g.gs) s = alpha > 0 ? c.take<int32_t>(N * 4) : nullptr;
    int32_t *queue_a = c.take<int32_t>(N * 4);
    int32_t *queue_b = c.take<int32_t>(N * 4);
    unsigned *visit = c.take<unsigned>((N + 31) / 32 * 4);  // the relabel's visited bits (written by it)
    const size_t tiles = (size_t)pog::tile_count_max(g);
    const int shape = (opt && opt->tile_shape > 0 && opt->tile_shape < pog::kTileShapes) ? opt->tile_shape : 0;
    const int bu_ratio = !opt || opt->bfs_bottom_up_ratio == 0 ? 8 : (opt->bfs_bottom_up_ratio < 0 ? 0 : opt->bfs_bottom_up_ratio);
    int32_t *tile_lists = c.take<int32_t>(4 * tiles * 4);
    int32_t *tile_work = c.take<int32_t>(256);
    pog::BfsSync *sync = c.take<pog::BfsSync>(sizeof(pog::BfsSync));
    pog::DevCounters *uctr = c.take<pog::DevCounters>(sizeof(pog::DevCounters));
    unsigned int *gap_bits = c.take<unsigned int>(kGapLevels / 8);  // right after the union counters
    g.ctr = c.take<pog::DevCounters>(sizeof(pog::DevCounters));
    g.trace = nullptr;
    pog::Grid *vol_table = c.take<pog::Grid>(sizeof(pog::Grid));
    int *node_base = c.take<int>(2 * sizeof(int));
    int *tile_base = c.take<int>(2 * sizeof(int));
    pog::Batch b{};
    b.vols = vol_table;
    b.node_base = node_base;
    b.tile_base = tile_base;
    b.nvol = 1;
    b.n_total = (int)N;
    b.ctr = uctr;
    b.trace = nullptr;
    b.visit = visit;
    b.wait_limit = (opt && opt->test_wait_limit > 0) ? opt->test_wait_limit : 0;
    const int bases[2] = {0, (int)N};
    const int tbases[2] = {0, (int)pog::tile_count(g, shape)};

    // The array keeps the previous call's contents: clear what must start at zero.
    NA_TRY_CUDA(cudaMemcpyAsync(vol_table, &g, sizeof(g), cudaMemcpyHostToDevice, st));
    NA_TRY_CUDA(cudaMemcpyAsync(node_base, bases, sizeof(bases), cudaMemcpyHostToDevice, st));
    NA_TRY_CUDA(cudaMemcpyAsync(tile_base, tbases, sizeof(tbases), cudaMemcpyHostToDevice, st));
    NA_TRY_CUDA(cudaMemsetAsync(uctr, 0, sizeof(pog::DevCounters), st));
    NA_TRY_CUDA(cudaMemsetAsync(g.ctr, 0, sizeof(pog::DevCounters), st));
    NA_TRY_CUDA(cudaMemsetAsync(tile_lists, 0, 4 * tiles * 4, st));
    NA_TRY_CUDA(cudaMemsetAsync(tile_work, 0, 6 * sizeof(int32_t), st));
    NA_TRY_CUDA(pog::launch_build_i32(g, cost_dev, st));

    pog::DevCounters host[2];
    std::memset(host, 0, sizeof host);
    NA_TRY(read_counters(uctr, g.ctr, host, st));
    if (!(flags & POG_FLAG_NO_PREPUSH)) NA_TRY_CUDA(pog::launch_column_prepush(g, st));
    const bool soft = alpha > 0;
    long long serial = 0;
    for (int round = 0;; ++round) {
        NA_TRY_CUDA(cudaMemsetAsync(&uctr->active, 0, sizeof(host[0].active), st));
        NA_TRY_CUDA(pog::launch_global_relabel(b, &g, queue_a, queue_b, sync, bfs_blocks, bu_ratio, st));
        NA_TRY(read_counters(uctr, g.ctr, host, st));
        if (host[0].active == 0) break;
        if (round + 1 >= max_rounds) return POG_E_NOCONVERGE;
        for (int k = 0; k < sweeps; ++k) {
            if (flags & POG_FLAG_NODE_SWEEPS)
                NA_TRY_CUDA(pog::launch_sweep(b, queue_a, &sync->size[0], kNodeOps, st));
            else
                NA_TRY_CUDA(pog::launch_tile_sweep(b, &g, 0, soft, shape, tile_lists, (long long)tiles, tile_work,
                                                   serial, k == 0, tile_sweeps, st));
            ++serial;
            if (!(flags & POG_FLAG_NO_GAP) && k + 1 == sweeps / 2) {
                NA_TRY_CUDA(cudaMemsetAsync(&uctr->max_label, 0, sizeof(int), st));
                NA_TRY_CUDA(pog::launch_gap(b, gap_bits, kGapLevels, st));
            }
        }
    }
    NA_TRY_CUDA(pog::launch_cut_reach(b, &g, queue_a, queue_b, sync, bfs_blocks, st));
    NA_TRY_CUDA(pog::launch_heights(g, heights_dev, st));
    NA_TRY_CUDA(cudaMemsetAsync(&g.ctr->excess_sum, 0, sizeof(host[1].excess_sum), st));
    NA_TRY_CUDA(pog::launch_excess_sum(g, st));
    NA_TRY(read_counters(uctr, g.ctr, host, st));
    *flow_out = (long long)host[1].bottom_const + (long long)host[1].src_total - (long long)host[1].excess_sum;
    return POG_OK;
}
