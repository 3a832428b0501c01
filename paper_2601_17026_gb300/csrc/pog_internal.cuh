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
    int changed;                     // a relaxation pass changed something
    int error;                       // POG_ERR_* bits
    int gap_level;                   // first empty label level found, or 0
    int max_label;                   // largest finite label seen
    int pad[4];
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
};

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

// Visit every residual arc u -> v of a non-bottom node u (the sink arc excluded):
// f(kind, d, v, residual). Residuals are read with L2-coherent loads.
template <bool SOFT, class F>
__device__ __forceinline__ void for_each_residual_arc(const Grid &g, int u, int x, int y, int z, F &&f) {
    if (z >= 2) {
        const int r = POG_CAP_INF - ldcg(g.fdn + u);
        if (r > 0) f(ARC_DOWN, 0, u - 1, r);
    }
    if (z + 1 < g.Z) {
        const int r = ldcg(g.fdn + u + 1);
        if (r > 0) f(ARC_UP, 0, u + 1, r);
    }
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        bool ok;
        const int off = nb_offset(g, x, y, d, ok);
        if (!ok) continue;
        if (z - g.delta >= 1) {
            const int r = POG_CAP_INF - ldcg(g.fh[d] + u);
            if (r > 0) f(ARC_HOUT, d, u + off - g.delta, r);
        }
        if (z + g.delta < g.Z) {
            const int v = u + off + g.delta;
            const int r = ldcg(g.fh[d ^ 1] + v);
            if (r > 0) f(ARC_HIN, d, v, r);
        }
        if (SOFT) {
            const int v = u + off;
            // d odd: towards x+1 / y+1, the pair lives at u; d even: it lives at v.
            const int r = (d & 1) ? g.alpha - ldcg(g.gs[d >> 1] + u) : g.alpha + ldcg(g.gs[d >> 1] + v);
            if (r > 0) f(ARC_SOFT, d, v, r);
        }
    }
}

}  // namespace pog

// Host-side graph object behind the opaque pog_graph handle.
struct pog_graph {
    int X, Y, Z, delta, alpha;
    long long N;
    cudaStream_t stream;
    void *arena;
    size_t arena_bytes;
    pog::Grid grid;
    int32_t *heights;            // device [X*Y]
    pog::DevCounters *ctr;       // device
    pog::DevCounters *ctr_host;  // pinned host mirror
    int solved;
    long long flow;
    int sweeps_per_relabel, max_rounds, tile_sweeps, flags;
    long long stats[8];
    // POG_FLAG_TIMING: event pairs per kernel family, folded into ms[] after a sync
    struct Timer {
        cudaEvent_t *ev = nullptr;
        int used = 0, cap = 0;
        double ms = 0.0;
    } timers[4];
};
