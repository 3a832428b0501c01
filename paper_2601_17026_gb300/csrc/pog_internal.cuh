// Internal definitions of the GB300 min-cut solver: device state, implicit addressing
// of the proper-order graph (Section 3.2.3) and the residual-arc enumeration shared by
// the push/relabel, global-relabel and cut kernels.
//
// Graph solved on the device. The bottom layer z = 0 of every column is always in the
// minimal minimum cut (its weights sum to -1 and every non-empty closed set contains
// it), so it is merged into the source s: arcs into it can never carry useful flow and
// are dropped, and its sink arcs add the constant sum_{z=0, w>0} w to the flow value.
// Remaining nodes: (x, y, z) with 1 <= z < Z. Arcs out of node u = (p, z):
//   sink   u -> t            residual snk[u]                 (w(u) > 0 initially)
//   down   u -> (p, z-1)     infinite, z >= 2                 flow fdn[u]
//   up     u -> (p, z+1)     reverse of (p,z+1)'s down arc    residual fdn[u+1]
//   hout_d u -> (q_d, z-D)   infinite, z-D >= 1              flow fh[d][u]
//   hin_d  u -> (q_d, z+D)   reverse of (q_d,z+D)'s arc in direction opp(d)
//                            residual fh[opp(d)][(q_d, z+D)]
//   soft_d u -> (q_d, z)     capacity alpha each way; the pair (p, p+x) keeps the net
//                            flow p -> p+x in gs[0][p], (p, p+y) in gs[1][p];
//                            residual alpha - g going up the axis, alpha + g going down.
// Directions d: 0 = x-1, 1 = x+1, 2 = y-1, 3 = y+1; opp(d) = d ^ 1.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define POG_INF 0x3fffffff       // label of a node that cannot reach the sink
#define POG_CAP_INF 0x7fffffff   // residual capacity standing in for an infinite arc

#define POG_ERR_COST_RANGE 1     // |c| >= 2^30 or a non-finite float cost
#define POG_ERR_FLOW_RANGE 2     // an infinite arc's flow or an excess reached int32 range
#define POG_ERR_TIMEOUT 4        // a bounded grid-barrier wait gave up

namespace pog {

struct DevCounters {
    unsigned long long src_total;    // sum over z >= 1 of max(-w, 0)
    unsigned long long bottom_sum;   // sum over columns of c(col, 0) (two's complement)
    unsigned long long pos_bottom;   // sum over columns other than (0,0) of max(c(col,0), 0)
    unsigned long long bottom_const; // sum over the bottom layer of max(w, 0)
    unsigned long long neg_bottom;   // sum over the bottom layer of max(-w, 0)
    unsigned long long neg_part;     // sum over columns other than (0,0) of max(-c(col,0), 0)
    unsigned long long excess_sum;   // sum of final excess over z >= 1
    unsigned long long active;       // active nodes (excess > 0, label < INF)
    unsigned long long raised;       // labels raised by the last gap relabel
    unsigned long long tiles_visited;  // tile visits of the tiled sweeps
    unsigned long long aug_offset;   // warm loss augmentation: what every cut gained (see k_augment)
    int changed;                     // a relaxation pass changed something
    int error;                       // POG_ERR_* bits
    int gap_level;                   // first empty label level found, or 0
    int max_label;                   // largest finite label seen
    int pad[4];
};

// Grid-barrier and frontier-size words of a cooperative BFS launch.
struct BfsSync {
    unsigned count;  // barrier arrivals since the launch
    unsigned gen;    // unused
    int size[3];     // frontier sizes, indexed by level mod 3
    int level1;      // nodes of level 1 (global relabel)
    int pad[2];
};

// Per-level trace of the last global relabel: frontier size, mode (0 top-down, 1
// bottom-up, 2 the pass that labels levels 1 and 2) and the device clock (ns) when the
// level started.
constexpr int kTraceLevels = 4096;
struct LevelTrace {
    long long size, mode, t_ns, pad;
};

struct Grid {
    int X, Y, Z, delta, alpha;
    int N;                 // X*Y*Z
    int32_t *lab;          // label (distance estimate to t); cut marks after extraction
    int32_t *exc;          // excess
    int32_t *snk;          // residual of the sink arc
    int32_t *fdn;          // flow on the down arc
    int32_t *fh[4];        // flow on the hard arcs, per direction
    int32_t *gs[2];        // net soft flow towards x+1 / y+1
    DevCounters *ctr;
    LevelTrace *trace;     // per-level trace of the global relabel (may be null)
    const void *tmap;      // device: tensor maps of the tile arrays (kTileArrays of them, in
                           // the order of the shared tile image), or null: plain tile loads
};

// Arrays of a shared-memory tile image, in image order: lab, exc, snk, fdn, fh[0..3],
// gs[0..1] (the last two only with soft arcs).
constexpr int kTileArrays = 10;
constexpr int kTensorMapBytes = 128;

// Volumes of a batch start at multiples of this many nodes in the union arrays, so every
// volume's arrays are 256-byte aligned (tensor-map and visited-bitmap word alignment).
constexpr int kNodeAlign = 64;

// A batch of independent volumes solved as one graph: the disjoint union of their
// graphs (they share only s and t), so one launch of each kernel serves all of them.
// Volume v owns union nodes [node_base[v], node_base[v+1]) and union tiles
// [tile_base[v], tile_base[v+1]); vols[v] views its slice of every union array. A single
// volume is a batch of one.
constexpr int kMaxVolumes = 1024;

struct Batch {
    const Grid *vols;      // device [nvol]
    const int *node_base;  // device [nvol + 1]
    const int *tile_base;  // device [nvol + 1] (tiles of the current tile shape)
    int nvol;
    int n_total;
    DevCounters *ctr;      // union counters: active nodes, BFS levels, gap, tile visits, timeouts
    LevelTrace *trace;     // per-level trace of the last global relabel (may be null)
    unsigned *visit;       // global relabel: one bit per union node, set once it is labelled
    int wait_limit;        // polls of a grid-barrier wait before it gives up (0: built-in limit)
};

// Largest v with base[v] <= idx (base ascending, base[0] = 0, nvol entries searched).
__device__ __forceinline__ int find_volume(const int *base, int nvol, int idx) {
    int lo = 0, hi = nvol - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base[mid] <= idx) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

enum ArcKind : int { ARC_NONE = -1, ARC_SINK = 0, ARC_DOWN, ARC_UP, ARC_HOUT, ARC_HIN, ARC_SOFT };

__device__ __forceinline__ int ldcg(const int32_t *p) { return __ldcg(p); }

// Neighbour column offset (in nodes) of direction d, or 0 with ok = false at the border.
__device__ __forceinline__ int nb_offset(const Grid &g, int x, int y, int d, bool &ok) {
    switch (d) {
        case 0: ok = x > 0;          return -g.Y * g.Z;
        case 1: ok = x + 1 < g.X;    return g.Y * g.Z;
        case 2: ok = y > 0;          return -g.Z;
        default: ok = y + 1 < g.Y;   return g.Z;
    }
}

// Gathered neighbourhood of a node: up to 14 arcs (2 vertical, 3 per direction) with
// their residual capacity and the far end's label, all loaded before any decision so
// the loads overlap instead of forming a dependent chain.
constexpr int kMaxArcs = 14;

struct Hood {
    int node[kMaxArcs];
    int res[kMaxArcs];   // residual capacity, 0 for an absent arc
    int lab[kMaxArcs];   // label (or mark) of the far end, POG_INF for an absent arc
};

// Loads of arc words: through L2 only while other threads may change them (sweeps), or
// through the read-only path when they are constant for the kernel (relabel, cut).
template <bool RO>
__device__ __forceinline__ int ld_arc(const int32_t *p) {
    return RO ? __ldg(p) : __ldcg(p);
}

// Infinite arcs: their forward residual is POG_CAP_INF minus their flow, and no flow
// reaches POG_CAP_INF without the solve failing with POG_E_OVERFLOW (every push checks),
// so in a search whose result is used they are always residual. INF_RES takes them so
// without loading their flow words (the searches that only need to know whether an arc
// is residual); the pushes, which need the amount, load it.

// Out-arcs of u: slot 0 down, 1 up, 2+3d hard out, 3+3d hard in (reverse), 4+3d soft.
// `far` (default: the labels) is the array read at each far end into h.lab.
template <bool SOFT, bool RO = false, bool INF_RES = false>
__device__ __forceinline__ void gather_out(const Grid &g, int u, int x, int y, int z, Hood &h,
                                           const int32_t *far = nullptr) {
#pragma unroll
    for (int i = 0; i < kMaxArcs; ++i) {
        h.res[i] = 0;
        h.node[i] = u;
    }
    if (z >= 2) {
        h.node[0] = u - 1;
        h.res[0] = INF_RES ? 1 : POG_CAP_INF - ld_arc<RO>(g.fdn + u);
    }
    if (z + 1 < g.Z) {
        h.node[1] = u + 1;
        h.res[1] = ld_arc<RO>(g.fdn + u + 1);
    }
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        bool ok;
        const int off = nb_offset(g, x, y, d, ok);
        if (!ok) continue;
        if (z - g.delta >= 1) {
            h.node[2 + 3 * d] = u + off - g.delta;
            h.res[2 + 3 * d] = INF_RES ? 1 : POG_CAP_INF - ld_arc<RO>(g.fh[d] + u);
        }
        if (z + g.delta < g.Z) {
            const int v = u + off + g.delta;
            h.node[3 + 3 * d] = v;
            h.res[3 + 3 * d] = ld_arc<RO>(g.fh[d ^ 1] + v);
        }
        if (SOFT) {
            const int v = u + off;
            h.node[4 + 3 * d] = v;
            h.res[4 + 3 * d] = (d & 1) ? g.alpha - ld_arc<RO>(g.gs[d >> 1] + u) : g.alpha + ld_arc<RO>(g.gs[d >> 1] + v);
        }
    }
    const int32_t *fv = far ? far : g.lab;
#pragma unroll
    for (int i = 0; i < kMaxArcs; ++i) h.lab[i] = ldcg(fv + h.node[i]);  // one round trip with the residuals
#pragma unroll
    for (int i = 0; i < kMaxArcs; ++i)
        if (h.res[i] <= 0) h.lab[i] = POG_INF;
}

// Out-arc slot k of u alone (slots as in gather_out): false when the arc is absent;
// else its far end and, when `want_res`, its residual capacity.
template <bool SOFT, bool RO = false>
__device__ __forceinline__ bool out_arc(const Grid &g, int u, int x, int y, int z, int k, bool want_res, int &node,
                                        int &res) {
    res = 0;
    if (k == 0) {
        node = u - 1;
        if (want_res && z >= 2) res = POG_CAP_INF - ld_arc<RO>(g.fdn + u);
        return z >= 2;
    }
    if (k == 1) {
        node = u + 1;
        if (want_res && z + 1 < g.Z) res = ld_arc<RO>(g.fdn + u + 1);
        return z + 1 < g.Z;
    }
    const int d = (k - 2) / 3, kind = (k - 2) % 3;
    bool ok;
    const int off = nb_offset(g, x, y, d, ok);
    if (kind == 0) {
        ok = ok && z - g.delta >= 1;
        node = u + off - g.delta;
        if (want_res && ok) res = POG_CAP_INF - ld_arc<RO>(g.fh[d] + u);
    } else if (kind == 1) {
        ok = ok && z + g.delta < g.Z;
        node = u + off + g.delta;
        if (want_res && ok) res = ld_arc<RO>(g.fh[d ^ 1] + node);
    } else {
        ok = ok && SOFT;
        node = u + off;
        if (want_res && ok)
            res = (d & 1) ? g.alpha - ld_arc<RO>(g.gs[d >> 1] + u) : g.alpha + ld_arc<RO>(g.gs[d >> 1] + node);
    }
    return ok;
}

// In-arcs of v (arcs u -> v): slot 0 from above, 1 from below, 2+3d hard arc of
// (q, z+D), 3+3d reverse of v's hard arc, 4+3d soft. With `visit`, h.lab receives the
// visited-bitmap word of each tail (union node base + u) instead of its label, all bits
// set for an absent arc.
template <bool SOFT, bool RO = false, bool INF_RES = false>
__device__ __forceinline__ void gather_in(const Grid &g, int v, int x, int y, int z, Hood &h,
                                          const unsigned *visit = nullptr, int base = 0) {
#pragma unroll
    for (int i = 0; i < kMaxArcs; ++i) {
        h.res[i] = 0;
        h.node[i] = v;
    }
    if (z + 1 < g.Z) {
        h.node[0] = v + 1;
        h.res[0] = INF_RES ? 1 : POG_CAP_INF - ld_arc<RO>(g.fdn + v + 1);
    }
    if (z >= 2) {
        h.node[1] = v - 1;
        h.res[1] = ld_arc<RO>(g.fdn + v);
    }
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        bool ok;
        const int off = nb_offset(g, x, y, d, ok);
        if (!ok) continue;
        if (z + g.delta < g.Z) {
            const int u = v + off + g.delta;
            h.node[2 + 3 * d] = u;
            h.res[2 + 3 * d] = INF_RES ? 1 : POG_CAP_INF - ld_arc<RO>(g.fh[d ^ 1] + u);
        }
        if (z - g.delta >= 1) {
            h.node[3 + 3 * d] = v + off - g.delta;
            h.res[3 + 3 * d] = ld_arc<RO>(g.fh[d] + v);
        }
        if (SOFT) {
            const int u = v + off;
            h.node[4 + 3 * d] = u;
            h.res[4 + 3 * d] = (d & 1) ? g.alpha + ld_arc<RO>(g.gs[d >> 1] + v) : g.alpha - ld_arc<RO>(g.gs[d >> 1] + u);
        }
    }
    if (visit) {
#pragma unroll
        for (int i = 0; i < kMaxArcs; ++i)
            h.lab[i] = ldcg(reinterpret_cast<const int32_t *>(visit) + ((base + h.node[i]) >> 5));
#pragma unroll
        for (int i = 0; i < kMaxArcs; ++i)
            if (h.res[i] <= 0) h.lab[i] = -1;
        return;
    }
#pragma unroll
    for (int i = 0; i < kMaxArcs; ++i) h.lab[i] = ldcg(g.lab + h.node[i]);
#pragma unroll
    for (int i = 0; i < kMaxArcs; ++i)
        if (h.res[i] <= 0) h.lab[i] = POG_INF;
}

}  // namespace pog

// Host-side graph object behind the opaque pog_graph handle: a batch of nvol volumes
// (one for pog_build) sharing one device arena.
struct pog_graph {
    int X, Y, Z, delta, alpha;   // volume 0 (the single-volume API)
    long long N;                 // nodes of volume 0
    int nvol;
    long long n_total;           // nodes of all volumes
    bool any_soft;
    cudaStream_t stream;
    void *arena;
    size_t arena_bytes;
    pog::Grid grid;              // view of volume 0
    pog::Grid *vols;             // host [nvol]: per-volume views
    pog::Grid *vols_dev;         // device [nvol]
    int *node_base, *tile_base;  // host [nvol + 1]
    int *node_base_dev, *tile_base_dev;
    long long *col_base;         // host [nvol + 1]: first column of each volume in `heights`
    pog::Batch batch;            // device-side batch view (all volumes)
    pog::Batch live;             // the volumes that still had active nodes at the last relabel
    pog::Grid *live_vols_dev;    // device [nvol]: tables of `live`
    int *live_node_base_dev, *live_tile_base_dev;
    pog::Grid *live_vols;        // host [nvol]
    int *live_node_base, *live_tile_base, *live_ids;  // host [nvol + 1]
    int nlive;
    int32_t *heights;            // device [sum of X*Y]
    int32_t *queue_a, *queue_b;  // device [n_total] each: BFS frontiers
    pog::BfsSync *bfs_sync;      // device: grid barrier + frontier sizes
    pog::LevelTrace *trace;      // device [kTraceLevels]: last global relabel
    int32_t *tiles;              // device [4][ntiles]: flag and list of two alternating sweep lists
    long long ntiles;
    int32_t *tile_work;          // device [6]: three (listed tiles, next tile to take) counter pairs
    long long tile_serial;       // tiled sweeps run so far (selects lists and counters)
    pog::DevCounters *ctr;       // device: union counters
    pog::DevCounters *vctr;      // device [nvol]: per-volume counters
    pog::DevCounters *ctr_host;  // pinned host mirror of ctr followed by vctr
    unsigned *visit;             // device [padded nodes / 32]: visited bits of the global relabel
    void *tmap_host;             // host [nvol][kTileArrays]: tensor maps of the tile arrays
    void *tmap_dev;              // device copy of tmap_host
    int solved;
    long long flow;              // volume 0
    long long *flows;            // host [nvol]
    int sweeps_per_relabel, max_rounds, tile_sweeps, flags, bfs_blocks;
    float relabel_factor;
    int tile_shape, bu_ratio;
    int wait_limit, fail_alloc;  // test hooks of pog_options
    cudaEvent_t round_ev[4];     // global relabel start/stop, sweep block start/stop
    long long stats[8];
    // POG_FLAG_TIMING: event pairs per kernel family, folded into ms[] after a sync
    struct Timer {
        cudaEvent_t *ev = nullptr;
        int used = 0, cap = 0;
        double ms = 0.0;
    } timers[4];
};
