// C ABI of the GB300 min-cut solver (declared in include/pog.h) and its host driver:
// state allocation, the push/relabel <-> global-relabel iteration with its exact
// termination test (Section 3.2.4), cut extraction and the flow value. Every graph is a
// batch: one volume for pog_build, several for pog_solve_batch, solved as the disjoint
// union of their graphs by the same launches.
#include <cstddef>
#include <cstdlib>
#include <cstring>
#include <new>

#include "pog.h"
#include "pog_internal.cuh"
#include "pog_launch.h"

using pog::DevCounters;
using pog::Grid;

namespace {

constexpr int kGapLevels = 1 << 20;          // labels tracked by the gap bitmap
constexpr int kFirstSweeps = 16;             // sweeps before the first adaptive choice
constexpr int kMaxSweeps = 1024;             // most sweeps between two global relabels
constexpr float kRelabelFactor = 1.0f;       // sweep time per round / global relabel time
constexpr int kNodeOps = 4;                  // push/relabel operations per node in a node sweep
constexpr int kDefaultTileSweeps = 8;        // local sweeps per tile visit
constexpr int kDefaultMaxRounds = 1 << 20;   // global relabels before giving up
constexpr int kBottomUpRatio = 8;            // BFS level bottom-up when frontier * 8 > unlabelled nodes

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

pog_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return POG_OK;
    return e == cudaErrorMemoryAllocation ? POG_E_NOMEM : POG_E_CUDA;
}

#define POG_TRY_CUDA(expr)                                   \
    do {                                                     \
        const pog_status _s = from_cuda((expr));             \
        if (_s != POG_OK) return _s;                         \
    } while (0)

#define POG_TRY(expr)                                        \
    do {                                                     \
        const pog_status _s = (expr);                        \
        if (_s != POG_OK) return _s;                         \
    } while (0)

void set_options(pog_graph *g, const pog_options *opt) {
    g->sweeps_per_relabel = (opt && opt->sweeps_per_relabel > 0) ? opt->sweeps_per_relabel : 0;  // 0: adaptive
    g->max_rounds = (opt && opt->max_rounds > 0) ? opt->max_rounds : kDefaultMaxRounds;
    g->tile_sweeps = (opt && opt->tile_sweeps > 0) ? opt->tile_sweeps : kDefaultTileSweeps;
    g->flags = opt ? opt->flags : 0;
    g->bfs_blocks = (opt && opt->bfs_blocks_per_sm > 0) ? opt->bfs_blocks_per_sm : 0;
    g->relabel_factor = (opt && opt->relabel_factor > 0.0f) ? opt->relabel_factor : kRelabelFactor;
    g->tile_shape = (opt && opt->tile_shape > 0 && opt->tile_shape < pog::kTileShapes) ? opt->tile_shape : 0;
    g->bu_ratio = !opt || opt->bfs_bottom_up_ratio == 0 ? kBottomUpRatio
                                                         : (opt->bfs_bottom_up_ratio < 0 ? 0 : opt->bfs_bottom_up_ratio);
    g->wait_limit = (opt && opt->test_wait_limit > 0) ? opt->test_wait_limit : 0;
    g->fail_alloc = (opt && opt->test_fail_alloc > 0) ? opt->test_fail_alloc : 0;
}

template <class T>
pog_status reset_field(pog_graph *g, T DevCounters::*field) {
    const size_t off = (size_t)((char *)&(g->ctr->*field) - (char *)g->ctr);
    return from_cuda(cudaMemsetAsync((char *)g->ctr + off, 0, sizeof(T), g->stream));
}

// Union counters and every volume's counters to the pinned mirror, then the error words.
pog_status read_counters(pog_graph *g) {
    POG_TRY_CUDA(cudaMemcpyAsync(g->ctr_host, g->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, g->stream));
    POG_TRY_CUDA(cudaMemcpyAsync(g->ctr_host + 1, g->vctr, sizeof(DevCounters) * g->nvol, cudaMemcpyDeviceToHost,
                                 g->stream));
    POG_TRY_CUDA(cudaStreamSynchronize(g->stream));
    int err = 0;
    for (int v = 0; v <= g->nvol; ++v) err |= g->ctr_host[v].error;
    if (err & POG_ERR_TIMEOUT) return POG_E_TIMEOUT;
    if (err) return POG_E_OVERFLOW;
    return POG_OK;
}

const DevCounters &volume_counters(const pog_graph *g, int v) { return g->ctr_host[1 + v]; }

enum { ST_BFS = 2, ST_CUT = 3, ST_SWEEP = 1, ST_ROUNDS = 0, ST_GAPS = 4, ST_ACTIVE0 = 5, ST_LAUNCHES = 6 };
enum { TM_SWEEP = 0, TM_BFS = 1, TM_CUT = 2, TM_BUILD = 3 };

// Launch wrapped in a pair of CUDA events when POG_FLAG_TIMING is set.
template <class Launch>
cudaError_t timed(pog_graph *g, int family, Launch launch) {
    if (!(g->flags & POG_FLAG_TIMING)) return launch();
    pog_graph::Timer &t = g->timers[family];
    if (t.used + 2 > t.cap) {
        const int cap = t.cap ? 2 * t.cap : 256;
        cudaEvent_t *ev = static_cast<cudaEvent_t *>(std::realloc(t.ev, sizeof(cudaEvent_t) * cap));
        if (!ev) return cudaErrorMemoryAllocation;
        for (int i = t.cap; i < cap; ++i) {
            const cudaError_t e = cudaEventCreate(&ev[i]);
            if (e != cudaSuccess) {
                t.ev = ev;
                t.cap = i;
                return e;
            }
        }
        t.ev = ev;
        t.cap = cap;
    }
    cudaError_t e = cudaEventRecord(t.ev[t.used], g->stream);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(t.ev[t.used + 1], g->stream);
    if (e == cudaSuccess) t.used += 2;
    return e;
}

// Fold recorded event pairs into milliseconds (the stream must have been synchronised).
void fold_timers(pog_graph *g) {
    for (auto &t : g->timers) {
        for (int i = 0; i + 1 < t.used; i += 2) {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, t.ev[i], t.ev[i + 1]) == cudaSuccess) t.ms += ms;
        }
        t.used = 0;
    }
}

// Drop from `live` the volumes whose last relabel found no active node: a volume with none
// never changes again (no tile of it is listed, nothing pushes into it, it shares no arc
// with another volume), so later relabels, sweeps and gap passes skip it.
pog_status shrink_live(pog_graph *g) {
    int n = 0;
    bool changed = false;
    for (int i = 0; i < g->nlive; ++i) {
        const int v = g->live_ids[i];
        if (volume_counters(g, v).active == 0) {
            changed = true;
            continue;
        }
        g->live_ids[n] = v;
        g->live_vols[n] = g->vols[v];
        g->live_node_base[n] = g->node_base[v];
        g->live_tile_base[n] = g->tile_base[v];
        ++n;
    }
    if (!changed || n == 0) return POG_OK;
    g->nlive = n;
    POG_TRY_CUDA(cudaMemcpyAsync(g->live_vols_dev, g->live_vols, sizeof(Grid) * n, cudaMemcpyHostToDevice, g->stream));
    POG_TRY_CUDA(cudaMemcpyAsync(g->live_node_base_dev, g->live_node_base, sizeof(int) * n, cudaMemcpyHostToDevice,
                                 g->stream));
    POG_TRY_CUDA(cudaMemcpyAsync(g->live_tile_base_dev, g->live_tile_base, sizeof(int) * n, cudaMemcpyHostToDevice,
                                 g->stream));
    POG_TRY_CUDA(cudaStreamSynchronize(g->stream));  // the host tables are rewritten next round
    g->live.nvol = n;
    return POG_OK;
}

// Global relabel (exact reverse BFS from t, one cooperative launch for the live volumes)
// fused with the termination count; returns the number of active nodes.
pog_status global_relabel(pog_graph *g, long long &active) {
    POG_TRY(reset_field(g, &DevCounters::active));
    POG_TRY_CUDA(cudaEventRecord(g->round_ev[0], g->stream));
    POG_TRY_CUDA(timed(g, TM_BFS, [&] {
        return pog::launch_global_relabel(g->live, g->nlive == 1 ? &g->live_vols[0] : nullptr, g->queue_a,
                                          g->queue_b, g->bfs_sync, g->bfs_blocks, g->bu_ratio, g->stream);
    }));
    POG_TRY_CUDA(cudaEventRecord(g->round_ev[1], g->stream));
    g->stats[ST_LAUNCHES] += 1;
    POG_TRY(read_counters(g));
    g->stats[ST_BFS] += g->ctr_host->max_label;  // BFS levels of this relabel
    active = (long long)g->ctr_host->active;
    if (active > 0) POG_TRY(shrink_live(g));
    return POG_OK;
}

unsigned int *gap_bits(pog_graph *g) {
    // The bitmap sits after the union counters in the arena.
    return reinterpret_cast<unsigned int *>(reinterpret_cast<char *>(g->ctr) + align_up(sizeof(DevCounters), 256));
}

pog_status reset_live(pog_graph *g) {
    g->nlive = g->nvol;
    for (int v = 0; v < g->nvol; ++v) {
        g->live_ids[v] = v;
        g->live_vols[v] = g->vols[v];
        g->live_node_base[v] = g->node_base[v];
        g->live_tile_base[v] = g->tile_base[v];
    }
    g->live = g->batch;
    g->live.vols = g->live_vols_dev;
    g->live.node_base = g->live_node_base_dev;
    g->live.tile_base = g->live_tile_base_dev;
    POG_TRY_CUDA(cudaMemcpyAsync(g->live_vols_dev, g->live_vols, sizeof(Grid) * g->nvol, cudaMemcpyHostToDevice,
                                 g->stream));
    POG_TRY_CUDA(cudaMemcpyAsync(g->live_node_base_dev, g->live_node_base, sizeof(int) * g->nvol,
                                 cudaMemcpyHostToDevice, g->stream));
    POG_TRY_CUDA(cudaMemcpyAsync(g->live_tile_base_dev, g->live_tile_base, sizeof(int) * g->nvol,
                                 cudaMemcpyHostToDevice, g->stream));
    return POG_OK;
}

pog_status maxflow_impl(pog_graph *g) {
    std::memset(g->stats, 0, sizeof g->stats);
    POG_TRY(reset_live(g));
    g->stats[ST_LAUNCHES] = 2 * g->nvol;  // the builds
    for (int f = TM_SWEEP; f <= TM_CUT; ++f) g->timers[f].ms = 0.0;
    POG_TRY(read_counters(g));  // surfaces build errors (cost range)
    long long active = 0;
    if (!(g->flags & POG_FLAG_NO_PREPUSH)) {
        for (int v = 0; v < g->nvol; ++v) POG_TRY_CUDA(pog::launch_column_prepush(g->vols[v], g->stream));
        g->stats[ST_LAUNCHES] += g->nvol;
    }
    POG_TRY(global_relabel(g, active));
    g->stats[ST_ROUNDS] = 1;
    g->stats[ST_ACTIVE0] = active;
    const bool gap = !(g->flags & POG_FLAG_NO_GAP);
    // Sweeps per global relabel: fixed when requested; otherwise chosen each round so the
    // device time of the sweeps balances that of one global relabel, the GPU form of the
    // paper's rule of relabelling after a fixed factor of n discharges (Section 3.3).
    int sweeps = g->sweeps_per_relabel > 0 ? g->sweeps_per_relabel : kFirstSweeps;
    while (active > 0) {
        if (g->stats[ST_ROUNDS] >= g->max_rounds) return POG_E_NOCONVERGE;
        float gr_ms = 0.0f;
        cudaEventElapsedTime(&gr_ms, g->round_ev[0], g->round_ev[1]);
        const int half = sweeps / 2;
        POG_TRY_CUDA(cudaEventRecord(g->round_ev[2], g->stream));
        for (int k = 0; k < sweeps; ++k) {
            POG_TRY_CUDA(timed(g, TM_SWEEP, [&] {
                if (g->flags & POG_FLAG_NODE_SWEEPS)
                    return pog::launch_sweep(g->live, g->queue_a, &g->bfs_sync->size[0], kNodeOps, g->stream);
                const cudaError_t e = pog::launch_tile_sweep(
                    g->live, g->nlive == 1 ? &g->live_vols[0] : nullptr, g->live_tile_base[0], g->any_soft,
                    g->tile_shape, g->tiles, g->ntiles, g->tile_work, g->tile_serial, k == 0, g->tile_sweeps,
                    g->stream);
                ++g->tile_serial;
                return e;
            }));
            if (gap && k + 1 == half) {
                POG_TRY(reset_field(g, &DevCounters::raised));
                POG_TRY(reset_field(g, &DevCounters::max_label));
                POG_TRY_CUDA(pog::launch_gap(g->live, gap_bits(g), kGapLevels, g->stream));
                g->stats[ST_LAUNCHES] += 3;
                g->stats[ST_GAPS]++;
            }
        }
        POG_TRY_CUDA(cudaEventRecord(g->round_ev[3], g->stream));
        g->stats[ST_SWEEP] += sweeps;
        // node sweeps: collect + push per sweep; tiled: the tile kernel per sweep, and the
        // list reset + activity scan on the first sweep of the round
        g->stats[ST_LAUNCHES] += (g->flags & POG_FLAG_NODE_SWEEPS) ? 2 * sweeps : sweeps + 2;
        POG_TRY(global_relabel(g, active));
        g->stats[ST_ROUNDS]++;
        if (g->sweeps_per_relabel <= 0) {
            float sw_ms = 0.0f;
            cudaEventElapsedTime(&sw_ms, g->round_ev[2], g->round_ev[3]);
            const float per = sw_ms / (float)sweeps;
            float want = per > 0.0f ? g->relabel_factor * gr_ms / per : (float)kMaxSweeps;
            want = want < (float)kFirstSweeps ? (float)kFirstSweeps : (want > (float)kMaxSweeps ? (float)kMaxSweeps : want);
            sweeps = (int)want;
        }
    }
    // Maximum preflow reached: extract the minimal cut, the heights and the flow values.
    POG_TRY_CUDA(timed(g, TM_CUT, [&] {
        return pog::launch_cut_reach(g->batch, g->nvol == 1 ? &g->vols[0] : nullptr, g->queue_a, g->queue_b,
                                     g->bfs_sync, g->bfs_blocks, g->stream);
    }));
    for (int v = 0; v < g->nvol; ++v) {
        POG_TRY_CUDA(pog::launch_heights(g->vols[v], g->heights + g->col_base[v], g->stream));
        POG_TRY_CUDA(cudaMemsetAsync(&g->vctr[v].excess_sum, 0, sizeof(unsigned long long), g->stream));
        POG_TRY_CUDA(pog::launch_excess_sum(g->vols[v], g->stream));
    }
    g->stats[ST_LAUNCHES] += 1 + 2 * g->nvol;  // cut, heights and excess sums
    POG_TRY(read_counters(g));
    g->stats[ST_CUT] = g->ctr_host->max_label;  // BFS levels of the cut extraction
    for (int v = 0; v < g->nvol; ++v) {
        const DevCounters &c = volume_counters(g, v);
        g->flows[v] = (long long)c.bottom_const + (long long)c.src_total - (long long)c.excess_sum;
    }
    g->flow = g->flows[0];
    fold_timers(g);
    g->solved = 1;
    return POG_OK;
}

struct VolumeSpec {
    int X, Y, Z, delta, alpha;
};

bool valid_volume(const VolumeSpec &v) {
    return v.X >= 1 && v.Y >= 1 && v.Z >= 1 && v.delta >= 0 && v.alpha >= 0 && v.alpha < (1 << 30);
}

// Allocate a batch graph for `n` volumes and lay out its arena; `launch(v, grid, stream)`
// enqueues the build of volume v.
template <class Launch>
pog_status build_batch(int n, const VolumeSpec *spec, const pog_options *opt, void *stream, pog_graph **out,
                       Launch launch) {
    if (!out || n < 1 || n > pog::kMaxVolumes) return POG_E_INVALID;
    // Every volume starts at a multiple of kNodeAlign nodes in the union arrays (and in the
    // soft-arc arrays), so its arrays are aligned for bulk tensor copies and its visited
    // bits start on a word boundary; the padding nodes belong to no volume.
    long long total = 0, padded = 0, soft_padded = 0, cols = 0;
    for (int v = 0; v < n; ++v) {
        if (!valid_volume(spec[v])) return POG_E_INVALID;
        const long long N = (long long)spec[v].X * spec[v].Y * spec[v].Z;
        const long long Np = (N + pog::kNodeAlign - 1) / pog::kNodeAlign * pog::kNodeAlign;
        total += N;
        padded += Np;
        if (spec[v].alpha > 0) soft_padded += Np;
        cols += (long long)spec[v].X * spec[v].Y;
    }
    if (padded >= (1ll << 31) - 64) return POG_E_INVALID;
    pog_graph *g = new (std::nothrow) pog_graph();
    if (!g) return POG_E_NOMEM;
    g->nvol = n;
    g->X = spec[0].X;
    g->Y = spec[0].Y;
    g->Z = spec[0].Z;
    g->delta = spec[0].delta;
    g->alpha = spec[0].alpha;
    g->N = (long long)g->X * g->Y * g->Z;
    g->n_total = total;
    g->any_soft = soft_padded > 0;
    g->stream = static_cast<cudaStream_t>(stream);
    set_options(g, opt);
    g->vols = new (std::nothrow) Grid[n]();
    g->node_base = new (std::nothrow) int[n + 1];
    g->tile_base = new (std::nothrow) int[n + 1];
    g->col_base = new (std::nothrow) long long[n + 1];
    g->flows = new (std::nothrow) long long[n]();
    g->live_vols = new (std::nothrow) Grid[n]();
    g->live_node_base = new (std::nothrow) int[n + 1];
    g->live_tile_base = new (std::nothrow) int[n + 1];
    g->live_ids = new (std::nothrow) int[n + 1];
    if (!g->vols || !g->node_base || !g->tile_base || !g->col_base || !g->flows || !g->live_vols ||
        !g->live_node_base || !g->live_tile_base || !g->live_ids) {
        pog_free(g);
        return POG_E_NOMEM;
    }
    long long tiles = 0;
    g->node_base[0] = 0;
    g->tile_base[0] = 0;
    g->col_base[0] = 0;
    for (int v = 0; v < n; ++v) {
        Grid d{};
        d.X = spec[v].X;
        d.Y = spec[v].Y;
        d.Z = spec[v].Z;
        tiles += pog::tile_count(d, g->tile_shape);
        const int N = spec[v].X * spec[v].Y * spec[v].Z;
        g->node_base[v + 1] = g->node_base[v] + (N + pog::kNodeAlign - 1) / pog::kNodeAlign * pog::kNodeAlign;
        g->tile_base[v + 1] = (int)tiles;
        g->col_base[v + 1] = g->col_base[v] + (long long)spec[v].X * spec[v].Y;
    }
    const size_t per = align_up((size_t)padded * sizeof(int32_t), 256);
    const size_t per_soft = align_up((size_t)soft_padded * sizeof(int32_t), 256);
    const size_t visit = align_up((size_t)padded / 8, 256);
    const size_t tmaps = align_up((size_t)n * pog::kTileArrays * pog::kTensorMapBytes, 256);
    const size_t heights = align_up((size_t)cols * sizeof(int32_t), 256);
    const size_t ctr = align_up(sizeof(DevCounters), 256) + (size_t)kGapLevels / 8;
    const size_t vctr = align_up(sizeof(DevCounters) * n, 256);
    const size_t sync = align_up(sizeof(pog::BfsSync), 256);
    const size_t trace = sizeof(pog::LevelTrace) * pog::kTraceLevels;
    const size_t tile_bytes = align_up(sizeof(int32_t) * (size_t)tiles, 256);
    const size_t table = 2 * (align_up(sizeof(Grid) * n, 256) + 2 * align_up(sizeof(int) * (n + 1), 256));
    g->arena_bytes = per * (8 + 2) + 2 * per_soft + heights + ctr + vctr + sync + trace + 4 * tile_bytes + 256 + table +
                     visit + tmaps;
    cudaError_t e = g->fail_alloc == 1 ? cudaErrorMemoryAllocation : cudaMalloc(&g->arena, g->arena_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        g->arena = nullptr;
        pog_free(g);
        return e == cudaErrorMemoryAllocation ? POG_E_NOMEM : POG_E_CUDA;
    }
    g->tmap_host = g->fail_alloc == 2 ? nullptr : std::calloc((size_t)n * pog::kTileArrays, pog::kTensorMapBytes);
    if (!g->tmap_host) {
        pog_free(g);
        return POG_E_NOMEM;
    }
    e = g->fail_alloc == 3 ? cudaErrorMemoryAllocation
                           : cudaHostAlloc(reinterpret_cast<void **>(&g->ctr_host), sizeof(DevCounters) * (n + 1),
                                           cudaHostAllocDefault);
    if (e != cudaSuccess) {
        g->ctr_host = nullptr;
        pog_free(g);
        return POG_E_NOMEM;
    }
    for (auto &ev : g->round_ev) {
        if (cudaEventCreate(&ev) != cudaSuccess) {
            ev = nullptr;
            pog_free(g);
            return POG_E_CUDA;
        }
    }
    // ---- arena layout
    char *p = static_cast<char *>(g->arena);
    auto take = [&](size_t bytes) {
        char *r = p;
        p += bytes;
        return r;
    };
    int32_t *arr[8];
    for (auto &a : arr) a = reinterpret_cast<int32_t *>(take(per));
    int32_t *soft[2];
    for (auto &a : soft) a = reinterpret_cast<int32_t *>(take(per_soft));
    g->queue_a = reinterpret_cast<int32_t *>(take(per));
    g->queue_b = reinterpret_cast<int32_t *>(take(per));
    g->heights = reinterpret_cast<int32_t *>(take(heights));
    g->bfs_sync = reinterpret_cast<pog::BfsSync *>(take(sync));
    g->trace = reinterpret_cast<pog::LevelTrace *>(take(trace));
    g->tiles = reinterpret_cast<int32_t *>(take(4 * tile_bytes));
    g->ntiles = (long long)(tile_bytes / sizeof(int32_t));
    g->tile_serial = 0;
    g->tile_work = reinterpret_cast<int32_t *>(take(256));
    g->vctr = reinterpret_cast<DevCounters *>(take(vctr));
    g->vols_dev = reinterpret_cast<Grid *>(take(align_up(sizeof(Grid) * n, 256)));
    g->node_base_dev = reinterpret_cast<int *>(take(align_up(sizeof(int) * (n + 1), 256)));
    g->tile_base_dev = reinterpret_cast<int *>(take(align_up(sizeof(int) * (n + 1), 256)));
    g->live_vols_dev = reinterpret_cast<Grid *>(take(align_up(sizeof(Grid) * n, 256)));
    g->live_node_base_dev = reinterpret_cast<int *>(take(align_up(sizeof(int) * (n + 1), 256)));
    g->live_tile_base_dev = reinterpret_cast<int *>(take(align_up(sizeof(int) * (n + 1), 256)));
    g->ctr = reinterpret_cast<DevCounters *>(take(ctr));
    g->visit = reinterpret_cast<unsigned *>(take(visit));
    g->tmap_dev = take(tmaps);
    long long soft_off = 0;
    for (int v = 0; v < n; ++v) {
        Grid &gr = g->vols[v];
        const long long off = g->node_base[v];
        gr.X = spec[v].X;
        gr.Y = spec[v].Y;
        gr.Z = spec[v].Z;
        gr.delta = spec[v].delta;
        gr.alpha = spec[v].alpha;
        gr.N = spec[v].X * spec[v].Y * spec[v].Z;  // the padding after it belongs to no volume
        gr.lab = arr[0] + off;
        gr.exc = arr[1] + off;
        gr.snk = arr[2] + off;
        gr.fdn = arr[3] + off;
        for (int d = 0; d < 4; ++d) gr.fh[d] = arr[4 + d] + off;
        for (int k = 0; k < 2; ++k) gr.gs[k] = spec[v].alpha > 0 ? soft[k] + soft_off : nullptr;
        if (spec[v].alpha > 0) soft_off += g->node_base[v + 1] - g->node_base[v];
        gr.ctr = g->vctr + v;
        gr.trace = nullptr;
        char *host_maps = static_cast<char *>(g->tmap_host) + (size_t)v * pog::kTileArrays * pog::kTensorMapBytes;
        const bool maps = !(g->flags & POG_FLAG_NO_TMA) && !(g->flags & POG_FLAG_NODE_SWEEPS) &&
                          pog::encode_tile_maps(gr, g->tile_shape, host_maps);
        gr.tmap = maps ? static_cast<char *>(g->tmap_dev) + (size_t)v * pog::kTileArrays * pog::kTensorMapBytes
                       : nullptr;
    }
    g->grid = g->vols[0];
    g->batch.vols = g->vols_dev;
    g->batch.node_base = g->node_base_dev;
    g->batch.tile_base = g->tile_base_dev;
    g->batch.nvol = n;
    g->batch.n_total = (int)total;
    g->batch.ctr = g->ctr;
    g->batch.trace = g->trace;
    g->batch.visit = g->visit;
    g->batch.wait_limit = g->wait_limit;
    e = cudaMemcpyAsync(g->tmap_dev, g->tmap_host, (size_t)n * pog::kTileArrays * pog::kTensorMapBytes,
                        cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->vols_dev, g->vols, sizeof(Grid) * n, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->node_base_dev, g->node_base, sizeof(int) * (n + 1), cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->tile_base_dev, g->tile_base, sizeof(int) * (n + 1), cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->ctr, 0, sizeof(DevCounters), g->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->vctr, 0, sizeof(DevCounters) * n, g->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->tiles, 0, 4 * tile_bytes, g->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->tile_work, 0, 6 * sizeof(int32_t), g->stream);
    for (int v = 0; v < n && e == cudaSuccess; ++v)
        e = timed(g, TM_BUILD, [&] { return launch(v, g->vols[v], g->stream); });
    if (e != cudaSuccess) {
        pog_free(g);
        return from_cuda(e);
    }
    *out = g;
    return POG_OK;
}

template <class Launch>
pog_status build_one(int32_t X, int32_t Y, int32_t Z, int32_t delta, int32_t alpha, const pog_options *opt,
                     void *stream, pog_graph **out, Launch launch) {
    const VolumeSpec v{X, Y, Z, delta, alpha};
    return build_batch(1, &v, opt, stream, out, [&](int, const Grid &g, cudaStream_t st) { return launch(g, st); });
}

}  // namespace

extern "C" {

pog_status pog_build(const int32_t *cost_dev, int32_t X, int32_t Y, int32_t Z, int32_t delta, int32_t alpha,
                     const pog_options *opt, void *stream, pog_graph **out) {
    if (!cost_dev) return POG_E_INVALID;
    return build_one(X, Y, Z, delta, alpha, opt, stream, out,
                     [&](const Grid &g, cudaStream_t st) { return pog::launch_build_i32(g, cost_dev, st); });
}

pog_status pog_build_f32(const float *cost_dev, float scale, int32_t X, int32_t Y, int32_t Z, int32_t delta,
                         int32_t alpha, const pog_options *opt, void *stream, pog_graph **out) {
    if (!cost_dev || !(scale > 0.0f)) return POG_E_INVALID;
    return build_one(X, Y, Z, delta, alpha, opt, stream, out, [&](const Grid &g, cudaStream_t st) {
        return pog::launch_build_f32(g, cost_dev, scale, nullptr, 0, st);
    });
}

pog_status pog_build_f32_augmented(const float *cost_dev, float scale, const int32_t *h_aug_dev, int32_t margin,
                                   int32_t X, int32_t Y, int32_t Z, int32_t delta, int32_t alpha,
                                   const pog_options *opt, void *stream, pog_graph **out) {
    if (!cost_dev || !h_aug_dev || !(scale > 0.0f) || margin < 0 || margin >= (1 << 28)) return POG_E_INVALID;
    return build_one(X, Y, Z, delta, alpha, opt, stream, out, [&](const Grid &g, cudaStream_t st) {
        return pog::launch_build_f32(g, cost_dev, scale, h_aug_dev, margin, st);
    });
}

pog_status pog_energy(const pog_graph *g, int64_t *energy_out) {
    if (!g || !energy_out) return POG_E_INVALID;
    if (!g->solved) return POG_E_STATE;
    // max-flow = E*(h) + K with K = -1 - sum_col c(col,0) + sum_{w<0} (-w) (the cut of
    // the closed set below h, Eq. 6, after the weights telescope along each column).
    const DevCounters &c = volume_counters(g, 0);
    const long long K = -1 - (long long)c.bottom_sum + (long long)c.src_total + (long long)c.neg_bottom;
    *energy_out = g->flow - K;
    return POG_OK;
}

pog_status pog_surface_energy(const float *cost_dev, float scale, const int32_t *h_dev, int32_t B, int32_t X,
                              int32_t Y, int32_t Z, int32_t alpha, int64_t *energy_dev, void *stream) {
    if (!cost_dev || !h_dev || !energy_dev || !(scale > 0.0f) || B < 0 || X < 1 || Y < 1 || Z < 1 || alpha < 0)
        return POG_E_INVALID;
    if (B == 0) return POG_OK;
    return from_cuda(pog::launch_surface_energy(cost_dev, scale, h_dev, B, X, Y, Z, alpha,
                                                reinterpret_cast<long long *>(energy_dev),
                                                static_cast<cudaStream_t>(stream)));
}

pog_status pog_maxflow(pog_graph *g, int64_t *flow_out) {
    if (!g || !flow_out) return POG_E_INVALID;
    g->solved = 0;
    const pog_status s = maxflow_impl(g);
    if (s == POG_OK) *flow_out = g->flow;
    return s;
}

pog_status pog_surface(pog_graph *g, int32_t *heights_dev) {
    if (!g || !heights_dev) return POG_E_INVALID;
    if (!g->solved) return POG_E_STATE;
    return from_cuda(cudaMemcpyAsync(heights_dev, g->heights, sizeof(int32_t) * (size_t)g->X * g->Y,
                                     cudaMemcpyDeviceToDevice, g->stream));
}

pog_status pog_stats(const pog_graph *g, pog_stats_t *out) {
    if (!g || !out) return POG_E_INVALID;
    std::memset(out, 0, sizeof *out);
    out->rounds = g->stats[ST_ROUNDS];
    out->sweeps = g->stats[ST_SWEEP];
    out->bfs_passes = g->stats[ST_BFS];
    out->cut_passes = g->stats[ST_CUT];
    out->gaps = g->stats[ST_GAPS];
    out->active_initial = g->stats[ST_ACTIVE0];
    out->launches = g->stats[ST_LAUNCHES];
    out->tiles_visited = (long long)g->ctr_host->tiles_visited;
    out->nodes = g->n_total;
    out->state_bytes = (long long)g->arena_bytes;
    if (g->timers[TM_BUILD].used) {  // the build was timed; its events are complete after pog_maxflow
        if (cudaStreamSynchronize(g->stream) != cudaSuccess) return POG_E_CUDA;
        fold_timers(const_cast<pog_graph *>(g));
    }
    out->sweep_ms = g->timers[TM_SWEEP].ms;
    out->bfs_ms = g->timers[TM_BFS].ms;
    out->cut_ms = g->timers[TM_CUT].ms;
    out->build_ms = g->timers[TM_BUILD].ms;
    return POG_OK;
}

pog_status pog_export_state(const pog_graph *g, int32_t *excess, int32_t *sink, int32_t *fdown, int32_t *fhard,
                            int32_t *gsoft, int32_t *in_cut) {
    if (!g) return POG_E_INVALID;
    if (!g->solved) return POG_E_STATE;
    const size_t bytes = sizeof(int32_t) * (size_t)g->N;
    struct {
        int32_t *dst;
        const int32_t *src;
    } copies[10] = {{excess, g->grid.exc}, {sink, g->grid.snk}, {fdown, g->grid.fdn}, {in_cut, g->grid.lab}};
    int n = 4;
    for (int d = 0; d < 4; ++d) copies[n++] = {fhard ? fhard + d * g->N : nullptr, g->grid.fh[d]};
    if (g->alpha > 0)
        for (int k = 0; k < 2; ++k) copies[n++] = {gsoft ? gsoft + k * g->N : nullptr, g->grid.gs[k]};
    for (int i = 0; i < n; ++i)
        if (copies[i].dst)
            POG_TRY_CUDA(cudaMemcpyAsync(copies[i].dst, copies[i].src, bytes, cudaMemcpyDeviceToHost, g->stream));
    POG_TRY_CUDA(cudaStreamSynchronize(g->stream));
    return POG_OK;
}

pog_status pog_trace(const pog_graph *g, int64_t *out, int32_t max_levels, int32_t *levels_out) {
    if (!g || !out || max_levels < 0 || !levels_out) return POG_E_INVALID;
    const int n = max_levels < pog::kTraceLevels ? max_levels : pog::kTraceLevels;
    pog::LevelTrace *tmp = static_cast<pog::LevelTrace *>(std::malloc(sizeof(pog::LevelTrace) * (n ? n : 1)));
    if (!tmp) return POG_E_NOMEM;
    cudaError_t e = cudaMemcpyAsync(tmp, g->trace, sizeof(pog::LevelTrace) * n, cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) {
        std::free(tmp);
        return from_cuda(e);
    }
    int used = 0;
    for (int i = 0; i < n; ++i) {
        out[3 * i] = tmp[i].size;
        out[3 * i + 1] = tmp[i].mode;
        out[3 * i + 2] = tmp[i].t_ns;
        if (tmp[i].mode == -1) {
            used = i + 1;
            break;
        }
    }
    *levels_out = used;
    std::free(tmp);
    return POG_OK;
}

void pog_free(pog_graph *g) {
    if (!g) return;
    cudaStreamSynchronize(g->stream);
    for (auto &t : g->timers) {
        for (int i = 0; i < t.cap; ++i) cudaEventDestroy(t.ev[i]);
        std::free(t.ev);
    }
    for (auto ev : g->round_ev)
        if (ev) cudaEventDestroy(ev);
    if (g->arena) cudaFree(g->arena);
    if (g->ctr_host) cudaFreeHost(g->ctr_host);
    std::free(g->tmap_host);
    delete[] g->vols;
    delete[] g->node_base;
    delete[] g->tile_base;
    delete[] g->col_base;
    delete[] g->flows;
    delete[] g->live_vols;
    delete[] g->live_node_base;
    delete[] g->live_tile_base;
    delete[] g->live_ids;
    delete g;
}

const char *pog_strerror(pog_status s) {
    switch (s) {
        case POG_OK: return "ok";
        case POG_E_INVALID: return "invalid argument";
        case POG_E_OVERFLOW: return "value out of the int32 range (cost magnitude or arc flow)";
        case POG_E_NOMEM: return "out of memory";
        case POG_E_CUDA: return "CUDA runtime error";
        case POG_E_NOCONVERGE: return "iteration cap reached before convergence";
        case POG_E_TIMEOUT: return "bounded device wait timed out";
        case POG_E_STATE: return "call out of order";
    }
    return "unknown status";
}

pog_status pog_quantise(const float *in_dev, int32_t *out_dev, int64_t n, float scale, void *stream) {
    if (n < 0 || (n > 0 && (!in_dev || !out_dev)) || !(scale > 0.0f)) return POG_E_INVALID;
    if (n == 0) return POG_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int *err = nullptr;
    POG_TRY_CUDA(cudaMallocAsync(reinterpret_cast<void **>(&err), sizeof(int), st));
    int host_err = 0;
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = pog::launch_quantise(in_dev, out_dev, n, scale, err, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host_err, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(err, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return from_cuda(e);
    return host_err ? POG_E_OVERFLOW : POG_OK;
}

pog_status pog_backward(float *grad_dev, const int32_t *h_dev, const int32_t *h_target_dev, const int32_t *h_hat_dev,
                        const float *g_energy_dev, const float *g_hinge_dev, int32_t B, int32_t X, int32_t Y,
                        int32_t Z, void *stream) {
    if (!grad_dev || !h_dev || !g_energy_dev || B < 0 || X < 1 || Y < 1 || Z < 1) return POG_E_INVALID;
    if (g_hinge_dev && (!h_target_dev || !h_hat_dev)) return POG_E_INVALID;
    if (B == 0) return POG_OK;
    return from_cuda(pog::launch_backward(grad_dev, h_dev, h_target_dev, h_hat_dev, g_energy_dev, g_hinge_dev, B,
                                          X * Y, Z, static_cast<cudaStream_t>(stream)));
}

pog_status pog_solve_batch(int32_t n, const pog_volume *vols, const pog_options *opt, void *stream,
                           int64_t *flows_out, int32_t *const *heights_dev) {
    if (n < 0 || (n > 0 && (!vols || !flows_out || !heights_dev))) return POG_E_INVALID;
    if (n == 0) return POG_OK;
    if (n > pog::kMaxVolumes) return POG_E_INVALID;
    VolumeSpec *spec = new (std::nothrow) VolumeSpec[n];
    if (!spec) return POG_E_NOMEM;
    for (int i = 0; i < n; ++i) {
        if (!vols[i].cost_dev || !heights_dev[i]) {
            delete[] spec;
            return POG_E_INVALID;
        }
        spec[i] = VolumeSpec{vols[i].X, vols[i].Y, vols[i].Z, vols[i].delta, vols[i].alpha};
    }
    pog_graph *g = nullptr;
    pog_status s = build_batch(n, spec, opt, stream, &g, [&](int v, const Grid &gr, cudaStream_t st) {
        return pog::launch_build_i32(gr, vols[v].cost_dev, st);
    });
    delete[] spec;
    if (s != POG_OK) return s;
    s = maxflow_impl(g);
    if (s == POG_OK) {
        for (int i = 0; i < n && s == POG_OK; ++i) {
            flows_out[i] = g->flows[i];
            s = from_cuda(cudaMemcpyAsync(heights_dev[i], g->heights + g->col_base[i],
                                          sizeof(int32_t) * (size_t)vols[i].X * vols[i].Y, cudaMemcpyDeviceToDevice,
                                          g->stream));
        }
    }
    pog_free(g);  // synchronises the stream first
    return s;
}

pog_status pog_solve_batch_f32(int32_t B, const float *cost_dev, float scale, const int32_t *h_aug_dev,
                               int32_t margin, int32_t X, int32_t Y, int32_t Z, int32_t delta, int32_t alpha,
                               const pog_options *opt, void *stream, int64_t *flows_out, int64_t *energies_out,
                               int32_t *heights_dev) {
    if (B < 0 || (B > 0 && (!cost_dev || !flows_out || !heights_dev)) || !(scale > 0.0f)) return POG_E_INVALID;
    if (h_aug_dev && (margin < 0 || margin >= (1 << 28))) return POG_E_INVALID;
    if (B == 0) return POG_OK;
    if (B > pog::kMaxVolumes) return POG_E_INVALID;
    VolumeSpec *spec = new (std::nothrow) VolumeSpec[B];
    if (!spec) return POG_E_NOMEM;
    for (int i = 0; i < B; ++i) spec[i] = VolumeSpec{X, Y, Z, delta, alpha};
    const size_t vol = (size_t)X * Y * Z, cols = (size_t)X * Y;
    pog_graph *g = nullptr;
    pog_status s = build_batch(B, spec, opt, stream, &g, [&](int v, const Grid &gr, cudaStream_t st) {
        return pog::launch_build_f32(gr, cost_dev + v * vol, scale, h_aug_dev ? h_aug_dev + v * cols : nullptr,
                                     h_aug_dev ? margin : 0, st);
    });
    delete[] spec;
    if (s != POG_OK) return s;
    s = maxflow_impl(g);
    if (s == POG_OK) {
        for (int i = 0; i < B; ++i) {
            flows_out[i] = g->flows[i];
            if (energies_out) {
                const DevCounters &c = volume_counters(g, i);
                const long long K = -1 - (long long)c.bottom_sum + (long long)c.src_total + (long long)c.neg_bottom;
                energies_out[i] = g->flows[i] - K;
            }
        }
        s = from_cuda(cudaMemcpyAsync(heights_dev, g->heights, sizeof(int32_t) * cols * B, cudaMemcpyDeviceToDevice,
                                      g->stream));
    }
    pog_free(g);  // synchronises the stream first
    return s;
}

pog_status pog_solve_batch_f32_hinge(int32_t B, const float *cost_dev, float scale, const int32_t *h_target_dev,
                                     int32_t margin, int32_t X, int32_t Y, int32_t Z, int32_t delta, int32_t alpha,
                                     const pog_options *opt, void *stream, int64_t *energies_out,
                                     int64_t *aug_energies_out, int64_t *hinge_out, int64_t *flows_out,
                                     int64_t *aug_flows_out, int32_t *heights_dev, int32_t *h_hat_dev) {
    if (B < 0 || !(scale > 0.0f) || margin < 0 || margin >= (1 << 28)) return POG_E_INVALID;
    if (B > 0 && (!cost_dev || !h_target_dev || !energies_out || !hinge_out || !heights_dev || !h_hat_dev))
        return POG_E_INVALID;
    if (B == 0) return POG_OK;
    if (B > pog::kMaxVolumes) return POG_E_INVALID;
    VolumeSpec *spec = new (std::nothrow) VolumeSpec[B];
    if (!spec) return POG_E_NOMEM;
    for (int i = 0; i < B; ++i) spec[i] = VolumeSpec{X, Y, Z, delta, alpha};
    const size_t vol = (size_t)X * Y * Z, cols = (size_t)X * Y;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    pog_graph *g = nullptr;
    pog_status s = build_batch(B, spec, opt, stream, &g, [&](int v, const Grid &gr, cudaStream_t q) {
        return pog::launch_build_f32(gr, cost_dev + v * vol, scale, nullptr, 0, q);
    });
    if (s != POG_OK) {
        delete[] spec;
        return s;
    }
    long long *et = reinterpret_cast<long long *>(std::malloc(sizeof(long long) * B));
    if (!et) s = POG_E_NOMEM;
    // E(h_t) of every target on the quantised costs, first: a height outside [0, Z) is an
    // invalid argument. The relabel queue serves as scratch (the solves overwrite it later).
    if (s == POG_OK)
        s = from_cuda(pog::launch_surface_energy(cost_dev, scale, h_target_dev, B, X, Y, Z, alpha,
                                                 reinterpret_cast<long long *>(g->queue_a), st));
    if (s == POG_OK)
        s = from_cuda(cudaMemcpyAsync(et, g->queue_a, sizeof(long long) * B, cudaMemcpyDeviceToHost, st));
    if (s == POG_OK) s = from_cuda(cudaStreamSynchronize(st));
    for (int i = 0; s == POG_OK && i < B; ++i)
        if (et[i] == (long long)0x8000000000000000ull) s = POG_E_INVALID;
    // the energy solve
    if (s == POG_OK) s = maxflow_impl(g);
    if (s == POG_OK) {
        for (int i = 0; i < B; ++i) {
            const DevCounters &c = volume_counters(g, i);
            const long long K = -1 - (long long)c.bottom_sum + (long long)c.src_total + (long long)c.neg_bottom;
            energies_out[i] = g->flows[i] - K;
            if (flows_out) flows_out[i] = g->flows[i];
        }
        s = from_cuda(cudaMemcpyAsync(heights_dev, g->heights, sizeof(int32_t) * cols * B, cudaMemcpyDeviceToDevice, st));
    }
    // the loss-augmented solve: from the energy solve's final state (warm), or rebuilt
    const bool cold = opt && (opt->flags & POG_FLAG_COLD_HINGE);
    if (s == POG_OK && cold) {
        pog_free(g);
        g = nullptr;
        s = build_batch(B, spec, opt, stream, &g, [&](int v, const Grid &gr, cudaStream_t q) {
            return pog::launch_build_f32(gr, cost_dev + v * vol, scale, h_target_dev + v * cols, margin, q);
        });
    } else if (s == POG_OK) {
        for (int v = 0; v < B && s == POG_OK; ++v)
            s = from_cuda(pog::launch_augment(g->vols[v], cost_dev + v * vol, scale, h_target_dev + v * cols, margin,
                                              st));
    }
    if (s == POG_OK) s = maxflow_impl(g);
    if (s == POG_OK) {
        for (int i = 0; i < B; ++i) {
            const DevCounters &c = volume_counters(g, i);
            const long long K = -1 - (long long)c.bottom_sum + (long long)c.src_total + (long long)c.neg_bottom;
            const long long eaug = g->flows[i] - K;  // E'(h_hat), the augmented energy
            if (aug_energies_out) aug_energies_out[i] = eaug;
            if (aug_flows_out) aug_flows_out[i] = g->flows[i] - (cold ? 0 : (long long)c.aug_offset);
            // min_h [E(h) - margin * Hamming(h, h_t)] = E'(h_hat) - margin * X * Y
            hinge_out[i] = et[i] - (eaug - (long long)margin * (long long)cols);
        }
        s = from_cuda(cudaMemcpyAsync(h_hat_dev, g->heights, sizeof(int32_t) * cols * B, cudaMemcpyDeviceToDevice, st));
    }
    delete[] spec;
    std::free(et);
    pog_free(g);  // synchronises the stream first
    return s;
}

}  // extern "C"
