// pog_solve_convex: the general proper-order graph of Section 1.2 with convex pairwise
// costs over the edge interval, E(h) = sum_col c(col, h) + sum_pairs f(|h_p - h_q|),
// |h_p - h_q| <= delta. See include/pog.h for the contract.
//
// Graph on the device (bottom layer z = 0 merged into the source, as in the other
// kernels: arcs into it are dropped, its sink arcs add a constant to the flow value).
// Node u = (p, z), 1 <= z < Z, direction k (0: x-1, 1: x+1, 2: y-1, 3: y+1), q_k the
// neighbour column. Arcs out of u and the word that holds each one's state:
//   sink   u -> t                residual snk[u]
//   down   u -> (p, z-1)         infinite, z >= 2                   flow fdn[u]
//   up     u -> (p, z+1)         reverse of the down arc above      residual fdn[u+1]
//   hout_k u -> (q_k, z-D)       infinite, z-D >= 1                 flow fh[k][u]
//   hin_k  u -> (q_k, z+D)       reverse of that node's hout_{k^1}  residual fh[k^1][(q_k, z+D)]
//   s0_k   u -> (q_k, z)         capacity k_0 each way; the pair (p, p+x) keeps the net flow
//                                p -> p+x in gs[0][p], (p, p+y) in gs[1][p]
//   sout_kj u -> (q_k, z-d_j)    capacity k_{d_j}, z-d_j >= 1       flow fl[j][k][u]
//   sin_kj  u -> (q_k, z+d_j)    reverse of that node's sout_{k^1,j} residual fl[j][k^1][(q_k, z+d_j)]
// Layer j = 0.. nl-1 lists the drops d_j in 1..delta-1 whose capacity
// k_d = f(d+1) - 2 f(d) + f(d-1) is positive; d = 0 is the pair layer s0.
//
// The solve: node-parallel lock-free push/relabel sweeps over the compacted active nodes
// (each node pushes along a residual arc to its lowest neighbour, relabelling first when
// it is not above it: Section 2.1's operations with one thread per node), global
// relabelling by a reverse BFS from the sink, one launch per level with the frontier size
// read by the host every few levels (no kernel waits on another, so nothing can hang),
// termination when an exact relabel leaves no active node, then the minimal cut as the
// residual reach of the nodes that keep excess and the surface as its top per column.
#include <cooperative_groups.h>

#include <cstring>

#include "pog.h"
#include "pog_internal.cuh"
#include "pog_launch.h"

namespace cg = cooperative_groups;

namespace {

constexpr int kCvThreads = 256;
constexpr int kCvMaxLayers = POG_CONVEX_MAX_DELTA;
constexpr int kCvLevelBatch = 32;     // BFS levels launched between two host reads of the frontier size
constexpr int kCvOps = 4;             // push/relabel operations per active node and sweep
// Out-arc slots per lane in the push step, at most: 32 * kCvMaxPasses >= 3 + 4 * (3 + 2 * 31),
// the slots of a node with every layer d = 1..31 present.
constexpr int kCvMaxPasses = 9;
constexpr int kCvSweeps = 64;         // default sweeps per global relabel
constexpr int kCvMaxRounds = 1 << 12;

struct CvCounters {
    unsigned long long src_total;   // sum over z >= 1 of max(-w, 0)
    unsigned long long bottom_sum;  // sum over columns of c(col, 0) (two's complement)
    unsigned long long pos_part;    // sum over columns other than (0,0) of max(c(col,0), 0)
    unsigned long long neg_part;    // sum over columns other than (0,0) of max(-c(col,0), 0)
    unsigned long long excess_sum;  // sum of the final excess over z >= 1
    unsigned long long listed;      // active nodes listed for the push/relabel sweeps, summed
    int error;                      // POG_ERR_* bits
    int pad;
};

struct CGrid {
    int X, Y, Z, delta, N;
    int k0;                   // capacity of layer d = 0 (0: no such arcs)
    int nl;                   // layers d >= 1 with positive capacity
    int ld[kCvMaxLayers];     // their drops
    int lk[kCvMaxLayers];     // their capacities
    int32_t *lab, *exc, *snk, *fdn;
    int32_t *fh[4];
    int32_t *gs[2];
    int32_t *fl;              // [nl][4][N]
    CvCounters *ctr;
};

__device__ __forceinline__ int32_t *flp(const CGrid &g, int j, int k) {
    return g.fl + (size_t)(j * 4 + k) * (size_t)g.N;
}

// Neighbour column offset (in nodes) of direction k, ok = false at the border.
__device__ __forceinline__ int cv_nb(const CGrid &g, int x, int y, int k, bool &ok) {
    switch (k) {
        case 0: ok = x > 0;          return -g.Y * g.Z;
        case 1: ok = x + 1 < g.X;    return g.Y * g.Z;
        case 2: ok = y > 0;          return -g.Z;
        default: ok = y + 1 < g.Y;   return g.Z;
    }
}



// Arc slots. Out-arcs of u: slot 0 sink, 1 down, 2 up, then for direction k the P = 3 + 2 nl
// slots 3 + k P + r: r = 0 hout, 1 hin, 2 s0, 3 + 2j sout_j, 4 + 2j sin_j (S_out = 3 + 4 P).
// In-arcs v -> u: slot 0 from (p, z+1), 1 from (p, z-1), then 2 + k P + r: r = 0 the hout of
// (q, z+D), 1 the reverse of u's hout, 2 s0 from (q, z), 3 + 2j the sout_j of (q, z+d_j),
// 4 + 2j the reverse of u's sout_j (S_in = 2 + 4 P). A slot decodes to its far end v (-1:
// the sink) and its residual a + sgn * (*p), or a alone when p is null (infinite arcs in a
// search, which only asks whether an arc is residual: no infinite arc's flow reaches
// POG_CAP_INF without the solve failing with POG_E_OVERFLOW). False: no such arc.
__device__ __forceinline__ int cv_slots_per_dir(const CGrid &g) { return 3 + 2 * g.nl; }

// Column out-arcs of u: r = 0 sink, 1 down, 2 up.
template <bool LOAD_INF>
__device__ __forceinline__ bool cv_out_column(const CGrid &g, int u, int z, int r, int &v, const int32_t *&p, int &a,
                                              int &sgn) {
    if (r == 0) {
        p = g.snk + u;
        a = 0;
        return true;
    }
    if (r == 1) {
        if (z < 2) return false;
        v = u - 1;
        if (LOAD_INF) {
            p = g.fdn + u;
            a = POG_CAP_INF;
            sgn = -1;
        }
        return true;
    }
    if (z + 1 >= g.Z) return false;
    v = u + 1;
    p = g.fdn + u + 1;
    a = 0;
    return true;
}

// Out-arc of u by direction k and position r within it (k = -1: the column slots, r = 0
// sink, 1 down, 2 up).
template <bool LOAD_INF>
__device__ __forceinline__ bool cv_out_arc(const CGrid &g, int u, int x, int y, int z, int k, int r, int &v,
                                           const int32_t *&p, int &a, int &sgn) {
    p = nullptr;
    a = 1;
    sgn = 1;
    v = -1;
    if (k < 0) return cv_out_column<LOAD_INF>(g, u, z, r, v, p, a, sgn);
    bool ok;
    const int off = cv_nb(g, x, y, k, ok);
    if (!ok) return false;
    if (r == 0) {
        if (z - g.delta < 1) return false;
        v = u + off - g.delta;
        if (LOAD_INF) {
            p = g.fh[k] + u;
            a = POG_CAP_INF;
            sgn = -1;
        }
        return true;
    }
    if (r == 1) {
        if (z + g.delta >= g.Z) return false;
        v = u + off + g.delta;
        p = g.fh[k ^ 1] + v;
        a = 0;
        return true;
    }
    if (r == 2) {
        if (g.k0 == 0) return false;
        v = u + off;
        a = g.k0;
        if (k & 1) {
            p = g.gs[k >> 1] + u;
            sgn = -1;
        } else {
            p = g.gs[k >> 1] + v;
        }
        return true;
    }
    const int j = (r - 3) >> 1, d = g.ld[j];
    if (((r - 3) & 1) == 0) {
        if (z - d < 1) return false;
        v = u + off - d;
        p = flp(g, j, k) + u;
        a = g.lk[j];
        sgn = -1;
        return true;
    }
    if (z + d >= g.Z) return false;
    v = u + off + d;
    p = flp(g, j, k ^ 1) + v;
    a = 0;
    return true;
}

template <bool LOAD_INF>
__device__ __forceinline__ bool cv_out_slot(const CGrid &g, int u, int x, int y, int z, int s, int P, int &v,
                                            const int32_t *&p, int &a, int &sgn) {
    if (s < 3) return cv_out_arc<LOAD_INF>(g, u, x, y, z, -1, s, v, p, a, sgn);
    const int k = (s - 3) / P;
    return cv_out_arc<LOAD_INF>(g, u, x, y, z, k, (s - 3) - k * P, v, p, a, sgn);
}


__device__ __forceinline__ bool cv_in_slot(const CGrid &g, int u, int x, int y, int z, int s, int P, int &v,
                                           const int32_t *&p, int &a, int &sgn) {
    p = nullptr;
    a = 1;
    sgn = 1;
    if (s == 0) {  // down arc of (p, z+1): infinite
        if (z + 1 >= g.Z) return false;
        v = u + 1;
        return true;
    }
    if (s == 1) {  // up arc of (p, z-1), the reverse of u's down arc
        if (z < 2) return false;
        v = u - 1;
        p = g.fdn + u;
        a = 0;
        return true;
    }
    const int k = (s - 2) / P, r = (s - 2) - k * P;
    bool ok;
    const int off = cv_nb(g, x, y, k, ok);
    if (!ok) return false;
    if (r == 0) {  // hout_{k^1} of (q, z+D) lands on u: infinite
        if (z + g.delta >= g.Z) return false;
        v = u + off + g.delta;
        return true;
    }
    if (r == 1) {  // reverse of u's hout_k, from (q, z-D)
        if (z - g.delta < 1) return false;
        v = u + off - g.delta;
        p = g.fh[k] + u;
        a = 0;
        return true;
    }
    if (r == 2) {  // s0 of q towards p
        if (g.k0 == 0) return false;
        v = u + off;
        a = g.k0;
        if (k & 1) {
            p = g.gs[k >> 1] + u;
        } else {
            p = g.gs[k >> 1] + v;
            sgn = -1;
        }
        return true;
    }
    const int j = (r - 3) >> 1, d = g.ld[j];
    if (((r - 3) & 1) == 0) {  // sout_{k^1,j} of (q, z+d) lands on u
        if (z + d >= g.Z) return false;
        v = u + off + d;
        p = flp(g, j, k ^ 1) + v;
        a = g.lk[j];
        sgn = -1;
        return true;
    }
    if (z - d < 1) return false;  // reverse of u's sout_kj, from (q, z-d)
    v = u + off - d;
    p = flp(g, j, k) + u;
    a = 0;
    return true;
}

// Add a to the flow of an infinite arc; true when it reaches POG_CAP_INF.
__device__ __forceinline__ bool cv_add_inf(int32_t *p, int a) {
    const int old = atomicAdd(p, a);
    return (long long)old + a >= (long long)POG_CAP_INF;
}

// Push a units from u along out-slot s with far end v (-1: the sink).
__device__ __forceinline__ void cv_push(const CGrid &g, int u, int s, int P, int v, int a) {
    bool over = false;
    if (s == 0) {
        atomicSub(g.snk + u, a);
    } else if (s == 1) {
        over = cv_add_inf(g.fdn + u, a);
    } else if (s == 2) {
        atomicSub(g.fdn + u + 1, a);
    } else {
        const int k = (s - 3) / P, r = (s - 3) - k * P;
        if (r == 0) {
            over = cv_add_inf(g.fh[k] + u, a);
        } else if (r == 1) {
            atomicSub(g.fh[k ^ 1] + v, a);
        } else if (r == 2) {
            if (k & 1) atomicAdd(g.gs[k >> 1] + u, a);
            else atomicSub(g.gs[k >> 1] + v, a);
        } else {
            const int j = (r - 3) >> 1;
            if (((r - 3) & 1) == 0) atomicAdd(flp(g, j, k) + u, a);
            else atomicSub(flp(g, j, k ^ 1) + v, a);
        }
    }
    atomicSub(g.exc + u, a);
    if (v >= 0) {
        const int old = atomicAdd(g.exc + v, a);
        if ((long long)old + a > 0x7fffffffLL) over = true;
    }
    if (over) atomicOr(&g.ctr->error, POG_ERR_FLOW_RANGE);
}

// One warp-aggregated append of v to a queue.
__device__ __forceinline__ void cv_append(int *queue, int *size, int v) {
    cg::coalesced_group grp = cg::coalesced_threads();
    int base = 0;
    if (grp.thread_rank() == 0) base = atomicAdd(size, (int)grp.size());
    base = grp.shfl(base, 0);
    queue[base + (int)grp.thread_rank()] = v;
}

__device__ __forceinline__ unsigned long long cv_warp_sum(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of v added once into *dst (all threads of the block call it).
__device__ __forceinline__ void cv_block_add(unsigned long long v, unsigned long long *dst) {
    __shared__ unsigned long long part[kCvThreads / 32];
    v = cv_warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) part[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < kCvThreads / 32 ? part[lane] : 0ull;
        v = cv_warp_sum(v);
        if (lane == 0 && v != 0ull) atomicAdd(dst, v);
    }
}

// ----------------------------------------------------------------------------------
// Graph construction (Section 1.2): node weights w(z) = c(z) - c(z-1) become source
// excess (w < 0) or sink residual (w > 0); every flow word starts at zero (zeroed by the
// host); the bottom layer's weights only enter the constants.
// ----------------------------------------------------------------------------------
__global__ void __launch_bounds__(kCvThreads) k_cv_build(CGrid g, const int32_t *cost) {
    const int u = blockIdx.x * kCvThreads + threadIdx.x;
    unsigned long long src = 0, bsum = 0, bpos = 0, bneg = 0;
    int err = 0;
    if (u < g.N) {
        const int z = u % g.Z;
        const int c = cost[u];
        if (c >= (1 << 30) || c <= -(1 << 30)) err |= POG_ERR_COST_RANGE;
        int e = 0, s = 0;
        if (z == 0) {
            bsum = (unsigned long long)(long long)c;
            if (u != 0 && c > 0) bpos = (unsigned long long)c;
            if (u != 0 && c < 0) bneg = (unsigned long long)(-(long long)c);
        } else {
            const int cm = cost[u - 1];
            if (cm >= (1 << 30) || cm <= -(1 << 30)) err |= POG_ERR_COST_RANGE;
            const int w = c - cm;
            e = w < 0 ? -w : 0;
            s = w > 0 ? w : 0;
            src = (unsigned long long)e;
        }
        g.lab[u] = POG_INF;
        g.exc[u] = e;
        g.snk[u] = s;
    }
    if (err) atomicOr(&g.ctr->error, err);
    cv_block_add(src, &g.ctr->src_total);
    cv_block_add(bsum, &g.ctr->bottom_sum);
    cv_block_add(bpos, &g.ctr->pos_part);
    cv_block_add(bneg, &g.ctr->neg_part);
}

// Active nodes (z >= 1, excess > 0, finite label) appended to `list`.
__global__ void __launch_bounds__(kCvThreads) k_cv_collect(CGrid g, int *list, int *count) {
    const int u = blockIdx.x * kCvThreads + threadIdx.x;
    bool a = false;
    if (u < g.N && u % g.Z != 0) a = __ldcg(g.exc + u) > 0 && __ldcg(g.lab + u) < POG_INF;
    if (a) cv_append(list, count, u);
}

// Lock-free push/relabel over the listed nodes, one warp per node (each node listed once,
// so one lane at a time owns its excess decrease, its sink arc and its label). The lanes
// split the node's out-arc slots; a warp minimum picks the residual arc with the lowest
// far-end label (ties: the lowest slot). A node not above that label is relabelled to it
// + 1 (Section 2.1's relabel), then min(excess, residual) is pushed along the arc. A node
// whose residual arcs all lead to label POG_INF cannot reach the sink and takes that
// label. Stale reads are safe: every value another thread may change concurrently moves
// in the direction that makes the push smaller than allowed.
// PASSES = ceil(S_out / 32) slots per lane; each lane's slots are decoded into (direction,
// position) once, before the node loop.
template <int PASSES>
__global__ void __launch_bounds__(kCvThreads, 4) k_cv_push_relabel(CGrid g, const int *list, const int *count, int ops) {
    const int n = __ldcg(count);
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&g.ctr->listed, (unsigned long long)n);
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * kCvThreads + threadIdx.x) >> 5;
    const int nwarps = gridDim.x * (kCvThreads / 32);
    const int P = cv_slots_per_dir(g), S = 3 + 4 * P;
    int kk[PASSES], rq[PASSES];  // kk = -2: no slot; -1: column slot rq
#pragma unroll
    for (int t = 0; t < PASSES; ++t) {
        const int s = lane + 32 * t;
        kk[t] = s >= S ? -2 : (s < 3 ? -1 : (s - 3) / P);
        rq[t] = s < 3 ? s : (s - 3) - (kk[t] < 0 ? 0 : kk[t]) * P;
    }
    for (int i = warp; i < n; i += nwarps) {
        const int u = __ldcg(list + i);
        const int z = u % g.Z, col = u / g.Z;
        const int x = col / g.Y, y = col % g.Y;
        for (int op = 0; op < ops; ++op) {
            int e = 0, l = 0;
            if (lane == 0) {
                e = __ldcg(g.exc + u);
                l = __ldcg(g.lab + u);
            }
            e = __shfl_sync(0xffffffffu, e, 0);
            l = __shfl_sync(0xffffffffu, l, 0);
            if (e <= 0 || l >= POG_INF) break;
            // All residual words of this lane's slots first, then the far-end labels of the
            // residual ones: two rounds of independent loads instead of a chain per slot.
            int vv[PASSES], rr[PASSES];
#pragma unroll
            for (int t = 0; t < PASSES; ++t) {
                vv[t] = -2;
                rr[t] = 0;
                int v, a, sgn;
                const int32_t *p;
                if (kk[t] != -2 && cv_out_arc<true>(g, u, x, y, z, kk[t], rq[t], v, p, a, sgn)) {
                    vv[t] = v;
                    rr[t] = p ? a + sgn * __ldcg(p) : a;
                }
            }
            int ll[PASSES];
#pragma unroll
            for (int t = 0; t < PASSES; ++t)
                ll[t] = rr[t] <= 0 ? POG_INF : (vv[t] < 0 ? 0 : __ldcg(g.lab + vv[t]));
            int best = POG_INF, bs = -1, bv = -1, br = 0;
#pragma unroll
            for (int t = 0; t < PASSES; ++t)
                if (ll[t] < best) {
                    best = ll[t];
                    bs = lane + 32 * t;
                    bv = vv[t];
                    br = rr[t];
                }
            unsigned long long key = ((unsigned long long)(unsigned)best << 32) | (unsigned)bs;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long other = __shfl_xor_sync(0xffffffffu, key, o);
                key = other < key ? other : key;
            }
            const int wbest = (int)(key >> 32);
            const int wslot = (int)(unsigned)(key & 0xffffffffu);
            if (wbest >= POG_INF) {
                if (lane == 0) g.lab[u] = POG_INF;
                break;
            }
            if (bs == wslot) {  // the one lane that found the arc
                if (l <= wbest) g.lab[u] = wbest + 1;
                cv_push(g, u, wslot, P, bv, e < br ? e : br);
            }
            __syncwarp();
        }
    }
}

// Level 0 of the reverse BFS: nodes with a residual sink arc get label 1 and their visited
// bit; every other node gets label POG_INF and a clear bit. One warp writes one bitmap word
// (32 consecutive nodes).
__global__ void __launch_bounds__(kCvThreads) k_cv_relabel_init(CGrid g, unsigned *visit, int *q0, int *sizes) {
    const int u = blockIdx.x * kCvThreads + threadIdx.x;
    bool a = false;
    if (u < g.N) {
        a = u % g.Z != 0 && __ldcg(g.snk + u) > 0;
        g.lab[u] = a ? 1 : POG_INF;
    }
    const unsigned bits = __ballot_sync(0xffffffffu, a);
    if ((threadIdx.x & 31) == 0 && u < g.N) visit[u >> 5] = bits;
    if (a) cv_append(q0, sizes, u);
}

// Cut extraction, level 0: the nodes that keep excess (z >= 1) are reached.
__global__ void __launch_bounds__(kCvThreads) k_cv_cut_init(CGrid g, unsigned *visit, int *q0, int *sizes) {
    const int u = blockIdx.x * kCvThreads + threadIdx.x;
    const bool a = u < g.N && u % g.Z != 0 && __ldcg(g.exc + u) > 0;
    const unsigned bits = __ballot_sync(0xffffffffu, a);
    if ((threadIdx.x & 31) == 0 && u < g.N) visit[u >> 5] = bits;
    if (a) cv_append(q0, sizes, u);
}

// One BFS level, one thread per (frontier node, arc slot) of the frontier sizes[level % 3]
// in qin. REACH = false: in-arcs (reverse BFS from the sink; a tail not yet visited whose
// arc into the frontier is residual gets label level + 2). REACH = true: out-arcs (reach
// of the excess nodes). The visited bit is tested before the residual word is loaded and
// claimed by an atomic OR; new nodes go to qout / sizes[(level + 1) % 3]. The counter of
// the level after that is cleared here for it.
template <bool REACH>
__global__ void __launch_bounds__(kCvThreads) k_cv_level(CGrid g, unsigned *visit, const int *qin, int *qout,
                                                         int *sizes, int level) {
    if (blockIdx.x == 0 && threadIdx.x == 0) sizes[(level + 2) % 3] = 0;
    const int n = __ldcg(sizes + level % 3);
    int *nsize = sizes + (level + 1) % 3;
    const int P = cv_slots_per_dir(g);
    const int S = REACH ? 3 + 4 * P : 2 + 4 * P;
    const long long total = (long long)n * S;
    const long long stride = (long long)gridDim.x * kCvThreads;
    for (long long i = (long long)blockIdx.x * kCvThreads + threadIdx.x; i < total; i += stride) {
        const int u = __ldcg(qin + i / S);
        const int s = (int)(i % S);
        const int z = u % g.Z, col = u / g.Z;
        const int x = col / g.Y, y = col % g.Y;
        int v, a, sgn;
        const int32_t *p;
        const bool ok = REACH ? (s != 0 && cv_out_slot<false>(g, u, x, y, z, s, P, v, p, a, sgn))
                              : cv_in_slot(g, u, x, y, z, s, P, v, p, a, sgn);
        if (!ok) continue;
        const unsigned bit = 1u << (v & 31);
        if (__ldcg(visit + (v >> 5)) & bit) continue;
        const int r = p ? a + sgn * __ldcg(p) : a;
        if (r <= 0) continue;
        if (atomicOr(visit + (v >> 5), bit) & bit) continue;
        if (!REACH) g.lab[v] = level + 2;
        cv_append(qout, nsize, v);
    }
}

// Sum of the final excess over z >= 1.
__global__ void __launch_bounds__(kCvThreads) k_cv_excess_sum(CGrid g) {
    const int u = blockIdx.x * kCvThreads + threadIdx.x;
    unsigned long long e = 0;
    if (u < g.N && u % g.Z != 0) {
        const int v = __ldcg(g.exc + u);
        e = v > 0 ? (unsigned long long)v : 0ull;
    }
    cv_block_add(e, &g.ctr->excess_sum);
}

// Surface: the top reached node of each column (0 when only the bottom layer is).
__global__ void __launch_bounds__(kCvThreads) k_cv_heights(CGrid g, const unsigned *visit, int32_t *heights) {
    const int col = blockIdx.x * kCvThreads + threadIdx.x;
    if (col >= g.X * g.Y) return;
    int h = 0;
    const long long base = (long long)col * g.Z;
    for (int z = g.Z - 1; z >= 1; --z) {
        const long long v = base + z;
        if ((__ldcg(visit + (v >> 5)) >> (v & 31)) & 1u) {
            h = z;
            break;
        }
    }
    heights[col] = h;
}

}  // namespace

// ----------------------------------------------------------------------------------
// Host driver
// ----------------------------------------------------------------------------------
namespace {

pog_status cv_status(cudaError_t e) { return e == cudaSuccess ? POG_OK : POG_E_CUDA; }

#define CV_TRY_CUDA(expr)                                  \
    do {                                                   \
        const pog_status _s = cv_status((expr));           \
        if (_s != POG_OK) return _s;                       \
    } while (0)
#define CV_TRY(expr)                                       \
    do {                                                   \
        const pog_status _s = (expr);                      \
        if (_s != POG_OK) return _s;                       \
    } while (0)

size_t cv_align(size_t v) { return (v + 255) / 256 * 256; }

int cv_blocks(long long n) { return (int)((n + kCvThreads - 1) / kCvThreads); }

// One solve's device buffers, launch shape and counters.
struct CvSolve {
    CGrid g{};
    cudaStream_t st = nullptr;
    void *arena = nullptr;
    int *qa = nullptr, *qb = nullptr, *list = nullptr, *count = nullptr, *sizes = nullptr;
    unsigned *visit = nullptr;          // one bit per node: visited by the current search
    pog::DevCounters *pctr = nullptr;   // error word of the column pre-push
    int persist_blocks = 0;         // grid of the grid-stride kernels: 8 blocks per SM
    bool timing = false;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    pog_stats_t stats{};
    CvCounters host_ctr{};
    int host_perr = 0;
    int host_int = 0;

    ~CvSolve() {
        if (arena) {
            cudaStreamSynchronize(st);
            cudaFree(arena);
        }
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }

    pog_status begin_timer() {
        if (timing) CV_TRY_CUDA(cudaEventRecord(ev[0], st));
        return POG_OK;
    }
    // Adds the time since begin_timer to *ms (synchronises the stream when timing).
    pog_status end_timer(double *ms) {
        if (!timing) return POG_OK;
        CV_TRY_CUDA(cudaEventRecord(ev[1], st));
        CV_TRY_CUDA(cudaEventSynchronize(ev[1]));
        float t = 0.f;
        CV_TRY_CUDA(cudaEventElapsedTime(&t, ev[0], ev[1]));
        *ms += t;
        return POG_OK;
    }

    pog_status read_int(const int *dev, int *out) {
        CV_TRY_CUDA(cudaMemcpyAsync(&host_int, dev, sizeof(int), cudaMemcpyDeviceToHost, st));
        CV_TRY_CUDA(cudaStreamSynchronize(st));
        *out = host_int;
        return POG_OK;
    }

    pog_status read_counters() {
        CV_TRY_CUDA(cudaMemcpyAsync(&host_ctr, g.ctr, sizeof(CvCounters), cudaMemcpyDeviceToHost, st));
        CV_TRY_CUDA(cudaMemcpyAsync(&host_perr, &pctr->error, sizeof(int), cudaMemcpyDeviceToHost, st));
        CV_TRY_CUDA(cudaStreamSynchronize(st));
        if (host_perr) return POG_E_OVERFLOW;
        if (host_ctr.error & POG_ERR_COST_RANGE) return POG_E_OVERFLOW;
        if (host_ctr.error & POG_ERR_FLOW_RANGE) return POG_E_OVERFLOW;
        if (host_ctr.error) return POG_E_CUDA;
        return POG_OK;
    }

    // Breadth-first levels from the frontier that `init` leaves in qa / sizes[0], until a
    // level finds nothing new; returns the number of levels run.
    template <bool REACH>
    pog_status levels(int64_t *nlevels) {
        int level = 0;
        for (;;) {
            for (int i = 0; i < kCvLevelBatch; ++i, ++level) {
                const int *qin = (level & 1) ? qb : qa;
                int *qout = (level & 1) ? qa : qb;
                k_cv_level<REACH><<<persist_blocks, kCvThreads, 0, st>>>(g, visit, qin, qout, sizes, level);
                CV_TRY_CUDA(cudaGetLastError());
                stats.launches++;
            }
            int n = 0;
            CV_TRY(read_int(sizes + level % 3, &n));
            if (n == 0) break;
        }
        *nlevels += level;
        return POG_OK;
    }

    pog_status global_relabel() {
        CV_TRY(begin_timer());
        CV_TRY_CUDA(cudaMemsetAsync(sizes, 0, 3 * sizeof(int), st));
        k_cv_relabel_init<<<cv_blocks(g.N), kCvThreads, 0, st>>>(g, visit, qa, sizes);
        CV_TRY_CUDA(cudaGetLastError());
        stats.launches++;
        CV_TRY(levels<false>(&stats.bfs_passes));
        return end_timer(&stats.bfs_ms);
    }

    // Active nodes into `list` / *count; returns their number.
    pog_status collect(bool read, int *active) {
        CV_TRY_CUDA(cudaMemsetAsync(count, 0, sizeof(int), st));
        k_cv_collect<<<cv_blocks(g.N), kCvThreads, 0, st>>>(g, list, count);
        CV_TRY_CUDA(cudaGetLastError());
        stats.launches++;
        if (read) CV_TRY(read_int(count, active));
        return POG_OK;
    }

    cudaError_t launch_push(const CGrid &gg, const int *l, const int *c) {
        const int passes = (3 + 4 * (3 + 2 * gg.nl) + 31) / 32;
        const dim3 grid(persist_blocks), block(kCvThreads);
        switch (passes) {
            case 1: k_cv_push_relabel<1><<<grid, block, 0, st>>>(gg, l, c, kCvOps); break;
            case 2: k_cv_push_relabel<2><<<grid, block, 0, st>>>(gg, l, c, kCvOps); break;
            case 3: k_cv_push_relabel<3><<<grid, block, 0, st>>>(gg, l, c, kCvOps); break;
            case 4: k_cv_push_relabel<4><<<grid, block, 0, st>>>(gg, l, c, kCvOps); break;
            case 5: k_cv_push_relabel<5><<<grid, block, 0, st>>>(gg, l, c, kCvOps); break;
            case 6: k_cv_push_relabel<6><<<grid, block, 0, st>>>(gg, l, c, kCvOps); break;
            case 7: k_cv_push_relabel<7><<<grid, block, 0, st>>>(gg, l, c, kCvOps); break;
            case 8: k_cv_push_relabel<8><<<grid, block, 0, st>>>(gg, l, c, kCvOps); break;
            default: k_cv_push_relabel<kCvMaxPasses><<<grid, block, 0, st>>>(gg, l, c, kCvOps); break;
        }
        return cudaGetLastError();
    }

    pog_status sweeps(int n) {
        CV_TRY(begin_timer());
        for (int s = 0; s < n; ++s) {
            if (s > 0) CV_TRY(collect(false, nullptr));
            CV_TRY_CUDA(launch_push(g, list, count));
            stats.launches++;
            stats.sweeps++;
        }
        return end_timer(&stats.sweep_ms);
    }

    pog_status cut(int32_t *heights) {
        CV_TRY(begin_timer());
        CV_TRY_CUDA(cudaMemsetAsync(sizes, 0, 3 * sizeof(int), st));
        k_cv_cut_init<<<cv_blocks(g.N), kCvThreads, 0, st>>>(g, visit, qa, sizes);
        CV_TRY_CUDA(cudaGetLastError());
        stats.launches++;
        CV_TRY(levels<true>(&stats.cut_passes));
        k_cv_heights<<<cv_blocks((long long)g.X * g.Y), kCvThreads, 0, st>>>(g, visit, heights);
        CV_TRY_CUDA(cudaGetLastError());
        k_cv_excess_sum<<<cv_blocks(g.N), kCvThreads, 0, st>>>(g);
        CV_TRY_CUDA(cudaGetLastError());
        stats.launches += 2;
        return end_timer(&stats.cut_ms);
    }
};

}  // namespace

extern "C" POG_API pog_status pog_solve_convex(const int32_t *cost_dev, int32_t X, int32_t Y, int32_t Z,
                                               int32_t delta, const int64_t *f_host, const pog_options *opt,
                                               void *stream, int64_t *flow_out, int64_t *energy_out,
                                               int32_t *heights_dev, pog_stats_t *stats_out) {
    if (!cost_dev || !flow_out || !heights_dev || X < 1 || Y < 1 || Z < 1 || delta < 0 ||
        delta > POG_CONVEX_MAX_DELTA || (delta > 0 && !f_host))
        return POG_E_INVALID;
    const long long N = (long long)X * Y * Z;
    if (N >= 0x7fffffffLL) return POG_E_INVALID;

    CvSolve s;
    CGrid &g = s.g;
    g.X = X;
    g.Y = Y;
    g.Z = Z;
    g.delta = delta;
    g.N = (int)N;
    // Layer capacities: k_0 = f(1), k_d = f(d+1) - 2 f(d) + f(d-1), f(0) = 0.
    for (int d = 0; d < delta; ++d) {
        const long long fd1 = f_host[d];
        const long long fd = d >= 1 ? f_host[d - 1] : 0;
        const long long fdm = d >= 2 ? f_host[d - 2] : 0;
        if (fd1 > (1LL << 40) || fd1 < -(1LL << 40)) return POG_E_INVALID;
        const long long k = d == 0 ? fd1 : fd1 - 2 * fd + fdm;
        if (k < 0 || k >= (1LL << 30)) return POG_E_INVALID;
        if (d == 0) {
            g.k0 = (int)k;
        } else if (k > 0) {
            g.ld[g.nl] = d;
            g.lk[g.nl] = (int)k;
            g.nl++;
        }
    }
    const int sweeps_per_round = opt && opt->sweeps_per_relabel > 0 ? opt->sweeps_per_relabel : kCvSweeps;
    const int max_rounds = opt && opt->max_rounds > 0 ? opt->max_rounds : kCvMaxRounds;
    s.timing = opt && (opt->flags & POG_FLAG_TIMING);
    s.st = static_cast<cudaStream_t>(stream);

    int dev = 0, sms = 0;
    CV_TRY_CUDA(cudaGetDevice(&dev));
    CV_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    s.persist_blocks = 8 * (sms > 0 ? sms : 1);
    if (s.timing) {
        CV_TRY_CUDA(cudaEventCreate(&s.ev[0]));
        CV_TRY_CUDA(cudaEventCreate(&s.ev[1]));
    }

    // Arena: counters, frontier sizes, then lab exc snk | fdn fh[4] gs[2] fl[nl][4] (the
    // flow words, zeroed in one memset) | qa qb list.
    const size_t arr = cv_align((size_t)N * 4);
    const int flow_arrays = 1 + 4 + 2 + 4 * g.nl;
    const size_t head = cv_align(sizeof(CvCounters)) + cv_align(4 * sizeof(int)) + cv_align(sizeof(pog::DevCounters));
    const size_t bits = cv_align(((size_t)N + 31) / 32 * 4);
    const size_t bytes = head + (3 + flow_arrays + 3) * arr + bits;
    if (opt && opt->test_fail_alloc == 1) return POG_E_NOMEM;
    if (cudaMalloc(&s.arena, bytes) != cudaSuccess) {
        s.arena = nullptr;
        cudaGetLastError();
        return POG_E_NOMEM;
    }
    char *p = static_cast<char *>(s.arena);
    g.ctr = reinterpret_cast<CvCounters *>(p);
    s.count = reinterpret_cast<int *>(p + cv_align(sizeof(CvCounters)));
    s.sizes = s.count + 1;
    s.pctr = reinterpret_cast<pog::DevCounters *>(p + cv_align(sizeof(CvCounters)) + cv_align(4 * sizeof(int)));
    p += head;
    auto take = [&]() {
        int32_t *r = reinterpret_cast<int32_t *>(p);
        p += arr;
        return r;
    };
    g.lab = take();
    g.exc = take();
    g.snk = take();
    char *flow_begin = p;
    g.fdn = take();
    for (int k = 0; k < 4; ++k) g.fh[k] = take();
    for (int k = 0; k < 2; ++k) g.gs[k] = take();
    // fl is indexed densely, fl + (j*4 + k) * N; its region of 4 * nl aligned arrays holds that.
    g.fl = reinterpret_cast<int32_t *>(p);
    p += (size_t)4 * g.nl * arr;
    const size_t flow_bytes = (size_t)(p - flow_begin);
    s.qa = take();
    s.qb = take();
    s.list = take();
    s.visit = reinterpret_cast<unsigned *>(p);
    p += bits;
    s.stats.nodes = N;
    s.stats.state_bytes = (long long)bytes;

    CV_TRY_CUDA(cudaMemsetAsync(s.arena, 0, head, s.st));
    CV_TRY_CUDA(cudaMemsetAsync(flow_begin, 0, flow_bytes, s.st));
    CV_TRY(s.begin_timer());
    k_cv_build<<<cv_blocks(N), kCvThreads, 0, s.st>>>(g, cost_dev);
    CV_TRY_CUDA(cudaGetLastError());
    s.stats.launches++;
    if (!(opt && (opt->flags & POG_FLAG_NO_PREPUSH))) {
        // Column pre-push along the infinite down arcs (the kernel of pog_build's solve, on a
        // view of this state: it touches only exc, snk and fdn, and the error word).
        pog::Grid view{};
        view.X = X;
        view.Y = Y;
        view.Z = Z;
        view.N = g.N;
        view.exc = g.exc;
        view.snk = g.snk;
        view.fdn = g.fdn;
        view.ctr = s.pctr;
        CV_TRY_CUDA(pog::launch_column_prepush(view, s.st));
        s.stats.launches++;
    }
    CV_TRY(s.end_timer(&s.stats.build_ms));
    CV_TRY(s.read_counters());
    int32_t c000 = 0;
    CV_TRY_CUDA(cudaMemcpyAsync(&c000, cost_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s.st));
    CV_TRY_CUDA(cudaStreamSynchronize(s.st));

    for (int round = 0;; ++round) {
        CV_TRY(s.global_relabel());
        s.stats.rounds++;
        int active = 0;
        CV_TRY(s.collect(true, &active));
        if (round == 0) s.stats.active_initial = active;
        CV_TRY(s.read_counters());
        if (active == 0) break;
        if (round + 1 >= max_rounds) {
            s.stats.tiles_visited = (long long)s.host_ctr.listed;
            if (stats_out) *stats_out = s.stats;
            return POG_E_NOCONVERGE;
        }
        CV_TRY(s.sweeps(sweeps_per_round));
    }
    CV_TRY(s.cut(heights_dev));
    CV_TRY(s.read_counters());

    const CvCounters &c = s.host_ctr;
    const long long w00 = (long long)c000 - 1 - (long long)c.bottom_sum;
    const long long bottom_const = (long long)c.pos_part + (w00 > 0 ? w00 : 0);
    const long long neg_bottom = (long long)c.neg_part + (w00 < 0 ? -w00 : 0);
    const long long flow = bottom_const + (long long)c.src_total - (long long)c.excess_sum;
    *flow_out = flow;
    if (energy_out) {
        const long long K = -1 - (long long)c.bottom_sum + (long long)c.src_total + neg_bottom;
        *energy_out = flow - K;
    }
    s.stats.tiles_visited = (long long)c.listed;
    if (stats_out) *stats_out = s.stats;
    return POG_OK;
}
