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

namespace cg = cooperative_groups;

namespace {

constexpr int kCvThreads = 256;
constexpr int kCvMaxLayers = POG_CONVEX_MAX_DELTA;
constexpr int kCvLevelBatch = 16;     // BFS levels launched between two host reads of the frontier size
constexpr int kCvOps = 4;             // push/relabel operations per active node and sweep
constexpr int kCvSweeps = 32;         // default sweeps per global relabel
constexpr int kCvMaxRounds = 1 << 12;
constexpr int kCvMark = -2;           // cut extraction: node reached

enum : int { CV_SINK = 0, CV_DOWN, CV_UP, CV_HOUT, CV_HIN, CV_S0, CV_SOUT, CV_SIN };

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

__device__ __forceinline__ int cv_slot(int kind, int k, int j) { return kind | (k << 4) | (j << 8); }

// Every out-arc of u: f(slot, head (-1 for t), residual). LOAD_INF: the residual of an
// infinite arc is POG_CAP_INF minus its flow (pushes need the amount); otherwise 1 (the
// searches only ask whether an arc is residual, and no infinite arc's flow reaches
// POG_CAP_INF without the solve failing with POG_E_OVERFLOW).
template <bool LOAD_INF, class F>
__device__ __forceinline__ void cv_out_arcs(const CGrid &g, int u, int x, int y, int z, F &&f) {
    f(CV_SINK, -1, __ldcg(g.snk + u));
    if (z >= 2) f(CV_DOWN, u - 1, LOAD_INF ? POG_CAP_INF - __ldcg(g.fdn + u) : 1);
    if (z + 1 < g.Z) f(CV_UP, u + 1, __ldcg(g.fdn + u + 1));
    for (int k = 0; k < 4; ++k) {
        bool ok;
        const int off = cv_nb(g, x, y, k, ok);
        if (!ok) continue;
        if (z - g.delta >= 1)
            f(cv_slot(CV_HOUT, k, 0), u + off - g.delta, LOAD_INF ? POG_CAP_INF - __ldcg(g.fh[k] + u) : 1);
        if (z + g.delta < g.Z) {
            const int v = u + off + g.delta;
            f(cv_slot(CV_HIN, k, 0), v, __ldcg(g.fh[k ^ 1] + v));
        }
        if (g.k0 > 0) {
            const int v = u + off;
            f(cv_slot(CV_S0, k, 0), v,
              (k & 1) ? g.k0 - __ldcg(g.gs[k >> 1] + u) : g.k0 + __ldcg(g.gs[k >> 1] + v));
        }
        for (int j = 0; j < g.nl; ++j) {
            const int d = g.ld[j];
            if (z - d >= 1) f(cv_slot(CV_SOUT, k, j), u + off - d, g.lk[j] - __ldcg(flp(g, j, k) + u));
            if (z + d < g.Z) {
                const int v = u + off + d;
                f(cv_slot(CV_SIN, k, j), v, __ldcg(flp(g, j, k ^ 1) + v));
            }
        }
    }
}

// Every in-arc v -> u of u: f(tail, residual of v -> u); infinite arcs report 1.
template <class F>
__device__ __forceinline__ void cv_in_arcs(const CGrid &g, int u, int x, int y, int z, F &&f) {
    if (z + 1 < g.Z) f(u + 1, 1);                        // down arc of (p, z+1)
    if (z >= 2) f(u - 1, __ldcg(g.fdn + u));             // reverse of u's down arc
    for (int k = 0; k < 4; ++k) {
        bool ok;
        const int off = cv_nb(g, x, y, k, ok);
        if (!ok) continue;
        if (z + g.delta < g.Z) f(u + off + g.delta, 1);  // hout_{k^1} of (q, z+D) lands on u
        if (z - g.delta >= 1) f(u + off - g.delta, __ldcg(g.fh[k] + u));  // reverse of u's hout_k
        if (g.k0 > 0) {
            const int v = u + off;
            f(v, (k & 1) ? g.k0 + __ldcg(g.gs[k >> 1] + u) : g.k0 - __ldcg(g.gs[k >> 1] + v));
        }
        for (int j = 0; j < g.nl; ++j) {
            const int d = g.ld[j];
            if (z + d < g.Z) {                           // sout_{k^1,j} of (q, z+d) lands on u
                const int v = u + off + d;
                f(v, g.lk[j] - __ldcg(flp(g, j, k ^ 1) + v));
            }
            if (z - d >= 1) f(u + off - d, __ldcg(flp(g, j, k) + u));  // reverse of u's sout_kj
        }
    }
}

// Add a to the flow of an infinite arc; true when it reaches POG_CAP_INF.
__device__ __forceinline__ bool cv_add_inf(int32_t *p, int a) {
    const int old = atomicAdd(p, a);
    return (long long)old + a >= (long long)POG_CAP_INF;
}

// Push a units from u along out-arc `slot` with head v (-1: the sink).
__device__ __forceinline__ void cv_push(const CGrid &g, int u, int slot, int v, int a) {
    const int kind = slot & 15, k = (slot >> 4) & 15, j = slot >> 8;
    bool over = false;
    switch (kind) {
        case CV_SINK: atomicSub(g.snk + u, a); break;
        case CV_DOWN: over = cv_add_inf(g.fdn + u, a); break;
        case CV_UP: atomicSub(g.fdn + u + 1, a); break;
        case CV_HOUT: over = cv_add_inf(g.fh[k] + u, a); break;
        case CV_HIN: atomicSub(g.fh[k ^ 1] + v, a); break;
        case CV_S0:
            if (k & 1) atomicAdd(g.gs[k >> 1] + u, a);
            else atomicSub(g.gs[k >> 1] + v, a);
            break;
        case CV_SOUT: atomicAdd(flp(g, j, k) + u, a); break;
        default: atomicSub(flp(g, j, k ^ 1) + v, a); break;  // CV_SIN
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

// Lock-free push/relabel over the listed nodes (each listed once, so one thread owns a
// node's excess decrease and its label): find the residual out-arc with the lowest head
// label; a node not above it is relabelled to that label + 1; then push
// min(excess, residual) along the arc. A node whose residual arcs all lead to label
// POG_INF cannot reach the sink and takes that label.
__global__ void __launch_bounds__(kCvThreads) k_cv_push_relabel(CGrid g, const int *list, const int *count, int ops) {
    const int n = __ldcg(count);
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&g.ctr->listed, (unsigned long long)n);
    for (int i = blockIdx.x * kCvThreads + threadIdx.x; i < n; i += gridDim.x * kCvThreads) {
        const int u = list[i];
        const int z = u % g.Z, col = u / g.Z;
        const int x = col / g.Y, y = col % g.Y;
        for (int op = 0; op < ops; ++op) {
            const int e = __ldcg(g.exc + u);
            int l = __ldcg(g.lab + u);
            if (e <= 0 || l >= POG_INF) break;
            int best = POG_INF, bslot = 0, bv = -1, br = 0;
            cv_out_arcs<true>(g, u, x, y, z, [&](int slot, int v, int r) {
                if (r <= 0) return;
                const int lv = v < 0 ? 0 : __ldcg(g.lab + v);
                if (lv < best) {
                    best = lv;
                    bslot = slot;
                    bv = v;
                    br = r;
                }
            });
            if (best >= POG_INF) {
                g.lab[u] = POG_INF;
                break;
            }
            if (l <= best) {
                l = best + 1;
                g.lab[u] = l;
            }
            cv_push(g, u, bslot, bv, e < br ? e : br);
        }
    }
}

// Level 0 of the reverse BFS: nodes with a residual sink arc get label 1.
__global__ void __launch_bounds__(kCvThreads) k_cv_relabel_init(CGrid g, int *q0, int *sizes) {
    const int u = blockIdx.x * kCvThreads + threadIdx.x;
    bool a = false;
    if (u < g.N) {
        a = u % g.Z != 0 && __ldcg(g.snk + u) > 0;
        g.lab[u] = a ? 1 : POG_INF;
    }
    if (a) cv_append(q0, sizes, u);
}

// Cut extraction, level 0: the nodes that keep excess (z >= 1) are reached; every other
// node is unmarked (label word 0).
__global__ void __launch_bounds__(kCvThreads) k_cv_cut_init(CGrid g, int *q0, int *sizes) {
    const int u = blockIdx.x * kCvThreads + threadIdx.x;
    bool a = false;
    if (u < g.N) {
        a = u % g.Z != 0 && __ldcg(g.exc + u) > 0;
        g.lab[u] = a ? kCvMark : 0;
    }
    if (a) cv_append(q0, sizes, u);
}

// One BFS level over the frontier sizes[level % 3] in qin: REACH = false expands in-arcs
// (reverse BFS from the sink: an unlabelled tail of a residual arc into the frontier gets
// label level + 2); REACH = true expands out-arcs (reach of the excess nodes: an unmarked
// head of a residual arc is marked). New nodes go to qout / sizes[(level + 1) % 3]; the
// counter of the level after that is cleared here for it.
template <bool REACH>
__global__ void __launch_bounds__(kCvThreads) k_cv_level(CGrid g, const int *qin, int *qout, int *sizes, int level) {
    if (blockIdx.x == 0 && threadIdx.x == 0) sizes[(level + 2) % 3] = 0;
    const int n = __ldcg(sizes + level % 3);
    int *nsize = sizes + (level + 1) % 3;
    const int free_word = REACH ? 0 : POG_INF;
    const int mark = REACH ? kCvMark : level + 2;
    for (int i = blockIdx.x * kCvThreads + threadIdx.x; i < n; i += gridDim.x * kCvThreads) {
        const int u = qin[i];
        const int z = u % g.Z, col = u / g.Z;
        const int x = col / g.Y, y = col % g.Y;
        auto claim = [&](int v, int r) {
            if (r <= 0 || __ldcg(g.lab + v) != free_word) return;
            if (atomicCAS(g.lab + v, free_word, mark) == free_word) cv_append(qout, nsize, v);
        };
        if (REACH) {
            cv_out_arcs<false>(g, u, x, y, z, [&](int, int v, int r) {
                if (v >= 0) claim(v, r);
            });
        } else {
            cv_in_arcs(g, u, x, y, z, claim);
        }
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
__global__ void __launch_bounds__(kCvThreads) k_cv_heights(CGrid g, int32_t *heights) {
    const int col = blockIdx.x * kCvThreads + threadIdx.x;
    if (col >= g.X * g.Y) return;
    int h = 0;
    const int32_t *lab = g.lab + (size_t)col * g.Z;
    for (int z = 1; z < g.Z; ++z)
        if (lab[z] == kCvMark) h = z;
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
    int persist_blocks = 0;         // grid of the grid-stride kernels: 8 blocks per SM
    bool timing = false;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    pog_stats_t stats{};
    CvCounters host_ctr{};
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
        CV_TRY_CUDA(cudaStreamSynchronize(st));
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
                k_cv_level<REACH><<<persist_blocks, kCvThreads, 0, st>>>(g, qin, qout, sizes, level);
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
        k_cv_relabel_init<<<cv_blocks(g.N), kCvThreads, 0, st>>>(g, qa, sizes);
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

    pog_status sweeps(int n) {
        CV_TRY(begin_timer());
        for (int s = 0; s < n; ++s) {
            if (s > 0) CV_TRY(collect(false, nullptr));
            k_cv_push_relabel<<<persist_blocks, kCvThreads, 0, st>>>(g, list, count, kCvOps);
            CV_TRY_CUDA(cudaGetLastError());
            stats.launches++;
            stats.sweeps++;
        }
        return end_timer(&stats.sweep_ms);
    }

    pog_status cut(int32_t *heights) {
        CV_TRY(begin_timer());
        CV_TRY_CUDA(cudaMemsetAsync(sizes, 0, 3 * sizeof(int), st));
        k_cv_cut_init<<<cv_blocks(g.N), kCvThreads, 0, st>>>(g, qa, sizes);
        CV_TRY_CUDA(cudaGetLastError());
        stats.launches++;
        CV_TRY(levels<true>(&stats.cut_passes));
        k_cv_heights<<<cv_blocks((long long)g.X * g.Y), kCvThreads, 0, st>>>(g, heights);
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
    const size_t head = cv_align(sizeof(CvCounters)) + cv_align(4 * sizeof(int));
    const size_t bytes = head + (3 + flow_arrays + 3) * arr;
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
    s.stats.nodes = N;
    s.stats.state_bytes = (long long)bytes;

    CV_TRY_CUDA(cudaMemsetAsync(s.arena, 0, head, s.st));
    CV_TRY_CUDA(cudaMemsetAsync(flow_begin, 0, flow_bytes, s.st));
    CV_TRY(s.begin_timer());
    k_cv_build<<<cv_blocks(N), kCvThreads, 0, s.st>>>(g, cost_dev);
    CV_TRY_CUDA(cudaGetLastError());
    s.stats.launches++;
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
        if (round + 1 >= max_rounds) return POG_E_NOCONVERGE;
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
