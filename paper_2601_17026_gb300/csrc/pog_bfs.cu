// Level-synchronous frontier BFS on the implicit residual graph, one cooperative launch
// per search: every level expands the current frontier queue into the next one, and the
// blocks meet at a grid barrier between levels (Section 3.2.2: the software barrier per
// level of the level-synchronised global relabel; Algorithm 3).
//
//   global relabel (reverse BFS from t): labels = exact residual distance to the sink,
//     INF where t is unreachable (which subsumes the gap heuristic at relabel time);
//     fused with the termination count of active nodes (Section 3.2.4).
//   cut extraction (forward BFS): marks = nodes reachable in the residual graph from the
//     nodes that hold excess, i.e. the source side of the minimal minimum cut.
//
// Frontier appends are warp-aggregated. In the global relabel a node joins a frontier
// once, through an atomicOr on its bit of a visited bitmap (one bit per node, 1/32 of the
// label array, so it stays in L2 while the labels do not); the cut extraction claims
// nodes by an atomicCAS on their mark. The grid barrier spins with an iteration limit; on
// timeout it raises POG_ERR_TIMEOUT and every block leaves.
#include <cooperative_groups.h>

#include "pog_internal.cuh"
#include "pog_launch.h"

namespace pog {

namespace {

// Each SM runs 1024 threads of a search grid, as 1, 2 or 4 blocks (fewer blocks: fewer
// arrivals at every grid barrier).
constexpr int kBfsSmThreads = 1024;
constexpr long long kBarrierSpinLimit = 1ll << 24;  // ~1-2 s of polling at worst

// Grid barrier over co-resident blocks on one monotonic arrival counter (zeroed before
// each launch): the k-th barrier is passed once the counter reaches k * nblocks. One
// atomic per block and a polling load, no second word to flip. False once the wait
// timed out (POG_ERR_TIMEOUT is raised and every block leaves).
__device__ __forceinline__ bool grid_sync(BfsSync *s, unsigned nblocks, int *err, int limit) {
    __syncthreads();
    __shared__ int ok;
    if (threadIdx.x == 0) {
        ok = 1;
        __threadfence();  // this block's writes before its arrival
        const unsigned old = atomicAdd(&s->count, 1u);
        const unsigned target = (old / nblocks + 1) * nblocks;
        const long long spin_limit = limit > 0 ? limit : kBarrierSpinLimit;
        long long spins = 0;
        while ((int)(*(volatile unsigned *)&s->count - target) < 0) {
            if (++spins > spin_limit || (*(volatile int *)err & POG_ERR_TIMEOUT)) {
                atomicOr(err, POG_ERR_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(20);
        }
        __threadfence();
    }
    __syncthreads();
    return ok;
}

// Append up to kMaxArcs nodes per thread (slot k of `hd.node` when bit k of `mask`) with one
// atomic per block: a frontier's size counter is shared by every block, and same-address
// atomics serialise, so one per warp made large levels wait on the counter. Every thread of
// the block must call it (the call holds two block barriers).
template <int K>
__device__ __forceinline__ void block_append_mask(unsigned mask, const int (&node)[K], int *queue, int *size) {
    __shared__ int warp_off[32];
    __shared__ int block_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cnt = __popc(mask);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_off[warp] = incl;  // the warp's total
    __syncthreads();
    if (threadIdx.x == 0) {
        int sum = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            const int t = warp_off[w];
            warp_off[w] = sum;
            sum += t;
        }
        block_base = sum ? atomicAdd(size, sum) : 0;
    }
    __syncthreads();
    int at = block_base + warp_off[warp] + incl - cnt;
#pragma unroll
    for (int k = 0; k < K; ++k)
        if (mask & (1u << k)) queue[at++] = node[k];
}

// Append `u` to a queue; the lanes that append together share one atomic.
__device__ __forceinline__ void warp_append(int u, int *queue, int *size) {
    namespace cg = cooperative_groups;
    const cg::coalesced_group grp = cg::coalesced_threads();
    int base = 0;
    if (grp.thread_rank() == 0) base = atomicAdd(size, (int)grp.size());
    base = grp.shfl(base, 0);
    queue[base + grp.thread_rank()] = u;
}

__device__ __forceinline__ void decode(const Grid &g, int u, int &x, int &y, int &z) {
    z = u % g.Z;
    const int col = u / g.Z;
    x = col / g.Y;
    y = col - x * g.Y;
}

// In-arcs of v with their residuals; h.lab receives the visited-bitmap word of each tail
// (union index base + node), or all bits set for an absent arc.
template <bool RO>
__device__ __forceinline__ void gather_in_any(const Grid &g, int v, int x, int y, int z, Hood &h,
                                              const unsigned *visit, int base) {
    if (g.gs[0]) gather_in<true, RO, true>(g, v, x, y, z, h, visit, base);
    else gather_in<false, RO, true>(g, v, x, y, z, h, visit, base);
}

// Out-arcs of u with their residuals (infinite arcs taken as residual without a load).
template <bool RO>
__device__ __forceinline__ void gather_out_any(const Grid &g, int u, int x, int y, int z, Hood &h,
                                               const int32_t *far = nullptr) {
    if (g.gs[0]) gather_out<true, RO, true>(g, u, x, y, z, h, far);
    else gather_out<false, RO, true>(g, u, x, y, z, h, far);
}

// Top-down expansion of frontier node v: claim, in the visited bitmap, every in-arc tail
// u (arc u -> v residual) not labelled yet; returns the mask of slots won (slots as in
// gather_in, tails in `node`, volume-local). The tails' bitmap words are read first (from
// L2); a residual word is then loaded only for an arc whose tail is still unvisited and
// whose residual is not known (infinite arcs are residual), so most of a node's scattered
// arc words are never fetched: in a search wave the greater part of the tails is already
// labelled.
template <bool SOFT>
__device__ __forceinline__ unsigned td_claim(const Grid &g, int v, int x, int y, int z, unsigned *visit, int base,
                                             int *node) {
    const int D = g.delta;
    unsigned exist = 0;
#pragma unroll
    for (int k = 0; k < kMaxArcs; ++k) node[k] = v;
    if (z + 1 < g.Z) {
        node[0] = v + 1;  // down arc of v+1 (infinite)
        exist |= 1u;
    }
    if (z >= 2) {
        node[1] = v - 1;  // up arc of v-1: residual fdn[v]
        exist |= 2u;
    }
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        bool ok;
        const int off = nb_offset(g, x, y, d, ok);
        if (!ok) continue;
        if (z + D < g.Z) {
            node[2 + 3 * d] = v + off + D;  // hard arc of (q, z+D) (infinite)
            exist |= 1u << (2 + 3 * d);
        }
        if (z - D >= 1) {
            node[3 + 3 * d] = v + off - D;  // reverse of v's hard arc: residual fh[d][v]
            exist |= 1u << (3 + 3 * d);
        }
        if (SOFT) {
            node[4 + 3 * d] = v + off;  // soft arc of (q, z)
            exist |= 1u << (4 + 3 * d);
        }
    }
    unsigned word[kMaxArcs];
#pragma unroll
    for (int k = 0; k < kMaxArcs; ++k)
        word[k] = (exist >> k & 1u) ? (unsigned)ldcg(reinterpret_cast<const int32_t *>(visit) + ((base + node[k]) >> 5))
                                    : 0xffffffffu;
    unsigned cand = 0;
#pragma unroll
    for (int k = 0; k < kMaxArcs; ++k) cand |= ((word[k] >> ((base + node[k]) & 31)) & 1u) ? 0u : 1u << k;
    if (!cand) return 0;
    int res[kMaxArcs];
#pragma unroll
    for (int k = 0; k < kMaxArcs; ++k) res[k] = 1;
    if (cand & 2u) res[1] = __ldg(g.fdn + v);
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        if (cand >> (3 + 3 * d) & 1u) res[3 + 3 * d] = __ldg(g.fh[d] + v);
        if (SOFT && (cand >> (4 + 3 * d) & 1u))
            res[4 + 3 * d] = (d & 1) ? g.alpha + __ldg(g.gs[d >> 1] + v) : g.alpha - __ldg(g.gs[d >> 1] + node[4 + 3 * d]);
    }
    unsigned old[kMaxArcs];
#pragma unroll
    for (int k = 0; k < kMaxArcs; ++k) {
        const int un = base + node[k];
        const unsigned bit = 1u << (un & 31);
        old[k] = ((cand >> k & 1u) && res[k] > 0) ? atomicOr(visit + (un >> 5), bit) : bit;
    }
    unsigned won = 0;
#pragma unroll
    for (int k = 0; k < kMaxArcs; ++k)
        if (!(old[k] & (1u << ((base + node[k]) & 31)))) won |= 1u << k;
    return won;
}

// Bottom-up test of an unlabelled node u: does one of its residual out-arcs end at a
// node of `level`? The far ends' labels are loaded first; residuals only for the arcs
// whose far end is at `level` (most nodes have none).
template <bool SOFT>
__device__ __forceinline__ bool bottom_up_hit(const Grid &g, int u, int x, int y, int z, int level) {
    int node[kMaxArcs];
    unsigned at = 0;
#pragma unroll
    for (int k = 0; k < kMaxArcs; ++k) {
        int r;
        if (out_arc<SOFT, true>(g, u, x, y, z, k, false, node[k], r)) at |= 1u << k;
    }
    int lab[kMaxArcs];
#pragma unroll
    for (int k = 0; k < kMaxArcs; ++k) lab[k] = (at >> k & 1u) ? ldcg(g.lab + node[k]) : POG_INF;
    unsigned cand = 0;
#pragma unroll
    for (int k = 0; k < kMaxArcs; ++k) cand |= (lab[k] == level ? 1u : 0u) << k;
    if (!cand) return false;
    bool hit = false;
#pragma unroll
    for (int k = 0; k < kMaxArcs; ++k) {
        if (!(cand >> k & 1u)) continue;
        int nd, r;
        out_arc<SOFT, true>(g, u, x, y, z, k, true, nd, r);
        hit |= r > 0;
    }
    return hit;
}

// Union node bases of the batch in shared memory (kMaxVolumes + 1 ints).
__device__ __forceinline__ void load_bases(const Batch &b, int *sbase) {
    for (int i = threadIdx.x; i <= b.nvol; i += blockDim.x) sbase[i] = b.node_base[i];
    __syncthreads();
}

template <bool SINGLE, int THREADS>
__global__ void __launch_bounds__(THREADS, kBfsSmThreads / THREADS) k_global_relabel(Batch b, Grid g0, int *qa, int *qb,
                                                                   BfsSync *sync, int bottom_up_ratio) {
    __shared__ int sbase[kMaxVolumes + 1];
    const unsigned nblocks = gridDim.x;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    int *err = &b.ctr->error;
    BfsSync *s = sync;
    load_bases(b, sbase);
    if (blockIdx.x == 0)  // per-volume termination counts, summed at the end
        for (int v = threadIdx.x; v < b.nvol; v += blockDim.x) b.vols[v].ctr->active = 0;
    long long unvisited = 0;
    unsigned long long t_start = 0;
    if (tid == 0 && b.trace) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_start));
    // levels 1 and 2 in one pass over the nodes: level 1 holds the nodes whose sink arc is
    // residual, level 2 the others with a residual arc into level 1 (read off the far
    // ends' sink residuals, which no step of the search changes); everything else starts
    // unreachable. Only level 2 is queued.
    // The warps cover aligned runs of 32 nodes (volume bases are multiples of 64 nodes), so
    // each writes whole words of the visited bitmap: bits of levels 1 and 2, and of the
    // bottom layer, which no search step may claim.
    int ones = 0;
    const int lane = threadIdx.x & 31;
    unsigned *visit = b.visit;
    for (int v = 0; v < b.nvol; ++v) {
        const Grid g = SINGLE ? g0 : b.vols[v];
        const int base = sbase[v];
        unvisited += (long long)g.N - (long long)g.X * g.Y;  // nodes z >= 1
        for (int ub = blockIdx.x * blockDim.x; ub < g.N; ub += stride) {  // block-uniform trip count
            const int u0 = ub + (threadIdx.x & ~31);
            const int u = u0 + lane;
            int l = POG_INF;
            bool bottom = false;
            if (u < g.N) {
                int x, y, z;
                decode(g, u, x, y, z);
                bottom = z == 0;
                if (!bottom) {
                    if (__ldg(g.snk + u) > 0) {
                        l = 1;
                    } else {
                        Hood hd;
                        gather_out_any<true>(g, u, x, y, z, hd, g.snk);
                        bool hit = false;
#pragma unroll
                        for (int k = 0; k < kMaxArcs; ++k) hit |= hd.res[k] > 0 && hd.lab[k] > 0;
                        if (hit) l = 2;
                    }
                }
                g.lab[u] = l;
            }
            const unsigned seen = __ballot_sync(0xffffffffu, bottom || l < POG_INF);
            if (lane == 0 && u0 < g.N) visit[(base + u0) >> 5] = seen;
            ones += l == 1;
            const int un[1] = {base + u};
            block_append_mask(l == 2 ? 1u : 0u, un, qb, &s->size[2]);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ones += __shfl_down_sync(0xffffffffu, ones, o);
    if ((threadIdx.x & 31) == 0 && ones) atomicAdd(&s->level1, ones);
    if (!grid_sync(s, nblocks, err, b.wait_limit)) return;
    unvisited -= *(volatile int *)&s->level1;
    if (tid == 0 && b.trace) b.trace[0] = LevelTrace{*(volatile int *)&s->level1, 2, (long long)t_start, 0};
    int level = 2;
    int *cur = qb, *nxt = qa;
    __shared__ int frontier;
    for (;;) {
        if (threadIdx.x == 0) frontier = *(volatile int *)&s->size[level % 3];
        __syncthreads();
        const int n = frontier;
        __syncthreads();
        if (n == 0) break;
        unvisited -= n;
        const bool bottom_up = bottom_up_ratio > 0 && (long long)n * bottom_up_ratio > unvisited;
        if (tid == 0) {
            s->size[(level + 2) % 3] = 0;  // level-1's counter, free again
            if (b.trace && level <= kTraceLevels) {
                unsigned long long t;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
                b.trace[level - 1] = LevelTrace{n, bottom_up ? 1 : 0, (long long)t, 0};
            }
        }
        if (bottom_up) {
            // bottom-up: every unlabelled node looks for a residual arc into this level;
            // neighbours sit at a fixed offset across a warp, so every load is coalesced
            for (int vi = 0; vi < b.nvol; ++vi) {
                const Grid g = SINGLE ? g0 : b.vols[vi];
                const int base = sbase[vi];
                for (int u0 = tid - lane; u0 < g.N; u0 += stride) {
                    const int u = u0 + lane;
                    const unsigned seen = ldcg(reinterpret_cast<const int32_t *>(visit) + ((base + u0) >> 5));
                    if (seen == 0xffffffffu) continue;  // the whole run is labelled (warp-uniform)
                    bool hit = false;
                    if (u < g.N && !((seen >> lane) & 1u)) {
                        int x, y, z;
                        decode(g, u, x, y, z);
                        hit = g.gs[0] ? bottom_up_hit<true>(g, u, x, y, z, level)
                                      : bottom_up_hit<false>(g, u, x, y, z, level);
                    }
                    const unsigned won = __ballot_sync(0xffffffffu, hit);
                    if (won && lane == 0) atomicOr(visit + ((base + u0) >> 5), won);
                    if (hit) {
                        g.lab[u] = level + 1;
                        warp_append(base + u, nxt, &s->size[(level + 1) % 3]);
                    }
                }
            }
        } else {
            // top-down: expand the frontier queue along residual arcs into its nodes; all
            // claims of a thread are issued together, appends cost one atomic per warp
            for (int first = blockIdx.x * blockDim.x; first < n; first += stride) {
                const int i = first + threadIdx.x;
                unsigned won = 0;
                Hood hd;
                int base = 0;
                if (i < n) {
                    const int uv = cur[i];
                    const int vi = SINGLE ? 0 : find_volume(sbase, b.nvol, uv);
                    // the volume's view read where used (a reference into the table),
                    // not copied whole into registers for every frontier node
                    const Grid &g = SINGLE ? g0 : b.vols[vi];
                    base = sbase[vi];
                    const int v = uv - base;
                    int x, y, z;
                    decode(g, v, x, y, z);
                    won = g.gs[0] ? td_claim<true>(g, v, x, y, z, visit, base, hd.node)
                                  : td_claim<false>(g, v, x, y, z, visit, base, hd.node);
#pragma unroll
                    for (int k = 0; k < kMaxArcs; ++k) {
                        if (won >> k & 1u) g.lab[hd.node[k]] = level + 1;
                        hd.node[k] += base;  // to union indices
                    }
                }
                block_append_mask(won, hd.node, nxt, &s->size[(level + 1) % 3]);
            }
        }
        if (!grid_sync(s, nblocks, err, b.wait_limit)) return;
        int *t = cur;
        cur = nxt;
        nxt = t;
        ++level;
    }
    if (tid == 0 && b.trace && level <= kTraceLevels) {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        b.trace[level - 1] = LevelTrace{0, -1, (long long)t, 0};
    }
    // termination test: active nodes (excess > 0 and a finite label), per volume and in all
    for (int vi = 0; vi < b.nvol; ++vi) {
        const Grid g = SINGLE ? g0 : b.vols[vi];
        unsigned long long active = 0;
        for (int u0 = tid; u0 < g.N; u0 += 4 * stride) {  // four independent excess loads in flight
            int e[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int u = u0 + j * stride;
                e[j] = (u < g.N && u % g.Z != 0) ? __ldcg(g.exc + u) : 0;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (e[j] < 0) atomicOr(err, POG_ERR_FLOW_RANGE);  // a wrapped excess
                if (e[j] > 0 && __ldcg(g.lab + u0 + j * stride) < POG_INF) ++active;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) active += __shfl_down_sync(0xffffffffu, active, o);
        if ((threadIdx.x & 31) == 0 && active) {
            atomicAdd(&g.ctr->active, active);
            atomicAdd(&b.ctr->active, active);
        }
    }
    if (tid == 0) b.ctr->max_label = level;
}

template <bool SINGLE, int THREADS>
__global__ void __launch_bounds__(THREADS, kBfsSmThreads / THREADS) k_cut_reach(Batch b, Grid g0, int *qa, int *qb, BfsSync *sync) {
    __shared__ int sbase[kMaxVolumes + 1];
    const unsigned nblocks = gridDim.x;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    int *err = &b.ctr->error;
    BfsSync *s = sync;
    load_bases(b, sbase);
    for (int vi = 0; vi < b.nvol; ++vi) {
        const Grid g = SINGLE ? g0 : b.vols[vi];
        const int base = sbase[vi];
        for (int u = tid; u < g.N; u += stride) {
            const bool seed = (u % g.Z != 0) && g.exc[u] > 0;
            g.lab[u] = seed ? 1 : 0;
            if (seed) warp_append(base + u, qa, &s->size[1]);
        }
    }
    if (!grid_sync(s, nblocks, err, b.wait_limit)) return;
    int level = 1;
    int *cur = qa, *nxt = qb;
    __shared__ int frontier;
    for (;;) {
        if (threadIdx.x == 0) frontier = *(volatile int *)&s->size[level % 3];
        __syncthreads();
        const int n = frontier;
        __syncthreads();
        if (n == 0) break;
        if (tid == 0) s->size[(level + 2) % 3] = 0;
        for (int first = blockIdx.x * blockDim.x; first < n; first += stride) {
            const int i = first + threadIdx.x;
            unsigned won = 0;
            Hood hd;
            if (i < n) {
                const int uv = cur[i];
                const int vi = SINGLE ? 0 : find_volume(sbase, b.nvol, uv);
                const Grid g = SINGLE ? g0 : b.vols[vi];
                const int base = sbase[vi];
                const int u = uv - base;
                int x, y, z;
                decode(g, u, x, y, z);
                gather_out_any<true>(g, u, x, y, z, hd);
                int old[kMaxArcs];
#pragma unroll
                for (int k = 0; k < kMaxArcs; ++k)
                    old[k] = (hd.res[k] > 0 && hd.lab[k] == 0) ? atomicCAS(g.lab + hd.node[k], 0, 1) : 1;
#pragma unroll
                for (int k = 0; k < kMaxArcs; ++k) {
                    if (hd.res[k] > 0 && hd.lab[k] == 0 && old[k] == 0) won |= 1u << k;
                    hd.node[k] += base;
                }
            }
            block_append_mask(won, hd.node, nxt, &s->size[(level + 1) % 3]);
        }
        if (!grid_sync(s, nblocks, err, b.wait_limit)) return;
        int *t = cur;
        cur = nxt;
        nxt = t;
        ++level;
    }
    if (tid == 0) b.ctr->max_label = level;
}

// Grid of a cooperative launch of `threads`-thread blocks: as many per SM as make
// 1024 threads, fewer if the occupancy calculator says they would not all be resident.
template <class K>
cudaError_t coop_blocks(K kernel, int threads, int &blocks) {
    int dev = 0, sms = 0, per_sm = 0, coop = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev)) != cudaSuccess) return e;
    if (!coop) return cudaErrorNotSupported;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0)) != cudaSuccess) return e;
    const int want = kBfsSmThreads / threads;
    blocks = sms * (per_sm < want ? per_sm : want);  // co-resident by construction
    return blocks < 1 ? cudaErrorInvalidConfiguration : cudaSuccess;
}

template <class K>
cudaError_t coop_launch(K kernel, int threads, void **args, BfsSync *sync, cudaStream_t st) {
    int blocks = 0;
    cudaError_t e = coop_blocks(kernel, threads, blocks);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(sync, 0, sizeof(BfsSync), st)) != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel(reinterpret_cast<void *>(kernel), blocks, threads, args, 0, st);
}

// Blocks per SM (1, 2 or 4; 0 and other values: 4) to the block size.
int bfs_threads(int blocks_per_sm) {
    return blocks_per_sm == 1 ? 1024 : (blocks_per_sm == 2 ? 512 : 256);
}

}  // namespace

cudaError_t launch_global_relabel(const Batch &b, const Grid *single, int *qa, int *qb, BfsSync *sync,
                                  int blocks_per_sm, int bottom_up_ratio, cudaStream_t st) {
    Batch bb = b;
    Grid g0 = single ? *single : Grid{};
    void *args[] = {&bb, &g0, &qa, &qb, &sync, &bottom_up_ratio};
    const int t = bfs_threads(blocks_per_sm);
    if (single) {
        if (t == 1024) return coop_launch(k_global_relabel<true, 1024>, t, args, sync, st);
        if (t == 512) return coop_launch(k_global_relabel<true, 512>, t, args, sync, st);
        return coop_launch(k_global_relabel<true, 256>, t, args, sync, st);
    }
    if (t == 1024) return coop_launch(k_global_relabel<false, 1024>, t, args, sync, st);
    if (t == 512) return coop_launch(k_global_relabel<false, 512>, t, args, sync, st);
    return coop_launch(k_global_relabel<false, 256>, t, args, sync, st);
}

cudaError_t launch_cut_reach(const Batch &b, const Grid *single, int *qa, int *qb, BfsSync *sync, int blocks_per_sm,
                             cudaStream_t st) {
    Batch bb = b;
    Grid g0 = single ? *single : Grid{};
    void *args[] = {&bb, &g0, &qa, &qb, &sync};
    const int t = bfs_threads(blocks_per_sm);
    if (single) {
        if (t == 1024) return coop_launch(k_cut_reach<true, 1024>, t, args, sync, st);
        if (t == 512) return coop_launch(k_cut_reach<true, 512>, t, args, sync, st);
        return coop_launch(k_cut_reach<true, 256>, t, args, sync, st);
    }
    if (t == 1024) return coop_launch(k_cut_reach<false, 1024>, t, args, sync, st);
    if (t == 512) return coop_launch(k_cut_reach<false, 512>, t, args, sync, st);
    return coop_launch(k_cut_reach<false, 256>, t, args, sync, st);
}

}  // namespace pog
