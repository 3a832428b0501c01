// Tiled push/relabel (Section 3.2.1's column segments, mapped to thread blocks): a block
// stages one tile of TX x TY columns x TZ heights of residual state in shared memory,
// runs several local push/relabel sweeps on it (Algorithm 2, lock-free in the manner of
// the node kernels), and stores its labels and sink residuals back. Only tiles holding an
// active node are visited.
//
// Ownership rules that keep concurrent tiles consistent:
//   * a node's label and sink residual change only in the tile that owns the node;
//   * every other word (excess, arc flows) may also be changed by neighbouring tiles, so
//     each push applies its changes both to the shared image (for this tile's later
//     reads) and to the global copy (by atomics that return nothing), exactly as a node
//     kernel would; nothing of these words is written back.
// Every residual capacity and excess a tile reads can only grow through other tiles'
// concurrent pushes (they add flow in the reverse direction, or excess), so a stale read
// never lets a tile push more than is there and the preflow stays valid, as in the node
// kernels; a stale label of a neighbour (too low) can cost convergence, never validity.
//
// Tile loads: when the volume has tensor maps (z extent a multiple of 4, arrays 16-byte
// aligned), one thread issues one bulk tensor copy (cp.async.bulk.tensor, TMA) per state
// array, a 3-D box of TX x TY x TZ int32 straight into the shared image, all completing on
// one mbarrier; out-of-volume box elements arrive as zeros and are then set to the values
// of a node outside the graph. Otherwise every thread loads its nodes' words one by one.
#include <cuda.h>

#include <cstring>

#include "pog_internal.cuh"
#include "pog_launch.h"

namespace pog {

namespace {

constexpr int kTileNodes = 1024;  // nodes per tile, every shape
constexpr int kTileThreads = 256;
constexpr int kPerThread = kTileNodes / kTileThreads;  // 4
constexpr int kTileBlocksPerSm = 4;                 // resident tile visits per SM
constexpr long long kTmaSpinLimit = 1ll << 22;      // polls of a tile load's mbarrier before giving up

// Tile shapes (columns in x, columns in y, heights), all of 1024 nodes. Node s of a tile
// sits at column c = s / TZ, height z0 + s % TZ, so consecutive threads read
// consecutive heights of one column (coalesced along z).
constexpr int kShapes[kTileShapes][3] = {{4, 8, 32}, {8, 8, 16}, {4, 4, 64}, {2, 4, 128}};

struct TileGeom {
    int tx, ty, tz;     // tile shape
    int ntx, nty, ntz;  // tiles per axis
};

TileGeom geom(const Grid &g, int shape) {
    const int *sh = kShapes[shape];
    return TileGeom{sh[0], sh[1], sh[2], (g.X + sh[0] - 1) / sh[0], (g.Y + sh[1] - 1) / sh[1],
                    (g.Z + sh[2] - 1) / sh[2]};
}

// Append tile t to a list once (its flag guards the membership).
__device__ __forceinline__ void list_tile(int t, int *flag, int *list, int *count) {
    if (__ldcg(flag + t)) return;
    if (atomicExch(flag + t, 1) == 0) list[atomicAdd(count, 1)] = t;
}

// List every tile (union numbering) that holds an active node, once. Each thread keeps
// four independent excess loads in flight.
__global__ void __launch_bounds__(256) k_collect_tiles(Batch b, int tx, int ty, int tz, int *flag, int *list,
                                                       int *count) {
    const int stride = gridDim.x * blockDim.x;
    for (int vi = 0; vi < b.nvol; ++vi) {
        const Grid g = b.vols[vi];
        const int tbase = b.tile_base[vi];
        const int nty = (g.Y + ty - 1) / ty, ntz = (g.Z + tz - 1) / tz;
        for (int u0 = blockIdx.x * blockDim.x + threadIdx.x; u0 < g.N; u0 += 4 * stride) {
            int e[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int u = u0 + j * stride;
                e[j] = u < g.N ? __ldcg(g.exc + u) : 0;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int u = u0 + j * stride;
                if (e[j] <= 0 || u % g.Z == 0 || __ldcg(g.lab + u) >= POG_INF) continue;
                const int z = u % g.Z;
                const int col = u / g.Z;
                const int x = col / g.Y, y = col - x * g.Y;
                list_tile(tbase + ((x / tx) * nty + (y / ty)) * ntz + z / tz, flag, list, count);
            }
        }
    }
}

// Unlist the tiles of one list (clear their flags) and empty it.
__global__ void __launch_bounds__(256) k_clear_listed(int *flag, const int *list, int *count) {
    const int n = *count;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) flag[list[i]] = 0;
}

// Shared-memory image of a tile, indexed by the node's place s in the tile. Every change
// a visit makes to a word that other tiles may also change (excess and arc words) is
// applied to the global copy at once as well (fire-and-forget atomics), so the image
// only serves reads; the owner-only words (label, sink residual) are stored at the end.
// The arrays follow one another in the order of the tensor maps (kTileArrays), each the
// target of one bulk tensor copy.
struct TileSmem {
    int lab[kTileNodes], exc[kTileNodes], snk[kTileNodes], fdn[kTileNodes];
    int fh[4][kTileNodes];
};
struct TileSoft {
    int gs[2][kTileNodes];
};
static_assert(sizeof(TileSmem) == 8 * 4 * kTileNodes, "tile image arrays must be contiguous");

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

// One bulk tensor copy of a 3-D box (coordinates z, y, x of its first element) into
// shared memory, completing on `bar` with its byte count.
__device__ __forceinline__ void tma_load_box(void *dst, const void *tmap, int z, int y, int x, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(tmap), "r"(z), "r"(y), "r"(x), "r"(smem_u32(bar))
        : "memory");
}

// Asynchronous copy of one 4-byte word from global to shared memory (through L1: every
// word a tile reads can only have grown since an older copy of its line was cached, so a
// stale read makes a push smaller, never invalid).
__device__ __forceinline__ void cp_async4(int *dst, const int32_t *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// Wait for phase `parity` of an mbarrier, with an iteration limit; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity) {
    const unsigned a = smem_u32(bar);
    for (long long i = 0; i < kTmaSpinLimit; ++i) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Lists of a tiled sweep: the tiles to visit now, and the next sweep's tiles (those a
// visit leaves active, and those that receive a push across their boundary).
struct TileLists {
    const int *list;  // this sweep's tiles
    const int *count;
    int *flag;        // membership in this sweep's list (cleared by each visit)
    int *next;        // work counter of this sweep
    int *nlist;       // next sweep's tiles
    int *ncount;
    int *nflag;
    int *zero;        // the counter pair of the sweep after next, zeroed here
};

// One visit of one tile: stage it in shared memory, run the local sweeps, write it back.
// `g` is the tile's volume, `tile` its union index (for the listing flags), `local_tile`
// its index within the volume.
// Returns false when the block must stop (a tile load's wait gave up; the error word is set).
template <int TX, int TY, int TZ, bool SOFT>
__device__ __forceinline__ bool tile_visit(const Grid &g, const Batch &b, int tile, int local_tile,
                                           const TileLists &L, int local_sweeps, TileSmem &S, TileSoft &SS,
                                           unsigned &nbmask, uint64_t *bar, unsigned &phase) {
    const bool soft = SOFT && g.gs[0] != nullptr;
    const int nty = (g.Y + TY - 1) / TY, ntz = (g.Z + TZ - 1) / TZ;
    const int tz = local_tile % ntz;
    const int txy = local_tile / ntz;
    const int x0 = (txy / nty) * TX, y0 = (txy % nty) * TY, z0 = tz * TZ;
    if (threadIdx.x == 0) {
        L.flag[tile] = 0;  // this sweep's listing is consumed
        nbmask = 0;
    }

    // ---- load (coalesced along z)
    // Node of tile place s, and whether the tile owns it (inside the volume, above the
    // bottom layer); recomputed where needed rather than kept live through the sweeps.
    auto node_of = [&](int s, bool &own) {
        const int c = s / TZ;  // column within the tile
        const int x = x0 + c / TY, y = y0 + c % TY, z = z0 + s % TZ;
        own = x < g.X && y < g.Y && z < g.Z && z >= 1;
        return (x * g.Y + y) * g.Z + z;
    };
    if (g.tmap) {
        // bulk tensor copies: one box per array, issued by one thread; the block waits on
        // the mbarrier (the previous visit's shared-memory accesses are ordered before the
        // copies' writes by the proxy fence after the block barrier that ended that visit)
        const int narr = soft ? kTileArrays : kTileArrays - 2;
        if (threadIdx.x == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                         "r"(narr * kTileNodes * 4)
                         : "memory");
            const char *maps = static_cast<const char *>(g.tmap);
            int *dst = S.lab;
#pragma unroll 1
            for (int a = 0; a < narr; ++a)
                tma_load_box(dst + a * kTileNodes, maps + a * kTensorMapBytes, z0, y0, x0, bar);
        }
        bool ok = mbar_wait(bar, phase);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) atomicOr(&g.ctr->error, POG_ERR_TIMEOUT);
            mbar_wait(bar, phase);  // let copies still in flight land before the block leaves
            return false;
        }
        phase ^= 1u;
#pragma unroll
        for (int k = 0; k < kPerThread; ++k) {
            const int s = threadIdx.x + kTileThreads * k;
            bool own;
            node_of(s, own);
            if (!own) {  // outside the volume, or the bottom layer: a node outside the graph
                S.lab[s] = POG_INF;
                S.exc[s] = 0;
                S.snk[s] = 0;
                S.fdn[s] = 0;
#pragma unroll
                for (int d = 0; d < 4; ++d) S.fh[d][s] = 0;
                if (soft) {
#pragma unroll
                    for (int j = 0; j < 2; ++j) SS.gs[j][s] = 0;
                }
            } else if (S.exc[s] < 0) {
                atomicOr(&g.ctr->error, POG_ERR_FLOW_RANGE);  // wrapped by small pushes
            }
        }
    } else {
        // word by word, as asynchronous 4-byte copies (no register staging, all in flight
        // together); a slot outside the graph gets its values by plain stores
#pragma unroll
        for (int k = 0; k < kPerThread; ++k) {
            const int s = threadIdx.x + kTileThreads * k;
            bool own;
            const int u = node_of(s, own);
            if (own) {
                cp_async4(S.lab + s, g.lab + u);
                cp_async4(S.exc + s, g.exc + u);
                cp_async4(S.snk + s, g.snk + u);
                cp_async4(S.fdn + s, g.fdn + u);
#pragma unroll
                for (int d = 0; d < 4; ++d) cp_async4(S.fh[d] + s, g.fh[d] + u);
                if (soft) {
#pragma unroll
                    for (int j = 0; j < 2; ++j) cp_async4(SS.gs[j] + s, g.gs[j] + u);
                }
            } else {
                S.lab[s] = POG_INF;
                S.exc[s] = 0;
                S.snk[s] = 0;
                S.fdn[s] = 0;
#pragma unroll
                for (int d = 0; d < 4; ++d) S.fh[d][s] = 0;
                if (soft) {
#pragma unroll
                    for (int j = 0; j < 2; ++j) SS.gs[j][s] = 0;
                }
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
#pragma unroll
        for (int k = 0; k < kPerThread; ++k)
            if (S.exc[threadIdx.x + kTileThreads * k] < 0)
                atomicOr(&g.ctr->error, POG_ERR_FLOW_RANGE);  // wrapped by small pushes
    }
    __syncthreads();

    // ---- local sweeps. Warps run them without block barriers (shared atomics keep
    // the tile consistent, and volatile reads see other warps' progress). In each sweep a
    // warp gathers its active nodes with ballots and steps them 32 at a time, so a sweep
    // costs in proportion to the active nodes; a warp stops once none of its nodes is
    // active. Arc slots: 0 down, 1 up, then per direction d (-x, +x, -y, +y): 2+3d the
    // hard arc out, 3+3d the reverse of the neighbour's hard arc, 4+3d the soft arc.
    volatile int *vexc = S.exc;
    volatile int *vlab = S.lab;
    const int lane = threadIdx.x & 31, wbase = threadIdx.x & ~31;
    const int X = g.X, Y = g.Y, Z = g.Z, D = g.delta;
    const int sx = Y * Z;
    for (int it = 0; it < local_sweeps; ++it) {
        unsigned m[kPerThread];
        int total = 0;
#pragma unroll
        for (int k = 0; k < kPerThread; ++k) {
            const int s = threadIdx.x + kTileThreads * k;
            m[k] = __ballot_sync(0xffffffffu, vexc[s] > 0 && vlab[s] < POG_INF);
            total += __popc(m[k]);
        }
        if (total == 0) break;
        for (int base = 0; base < total; base += 32) {
            // the r-th active node of the warp: its row k, then its lane (binary search)
            int r = base + lane;
            if (r >= total) continue;
            int k = 0;
            unsigned v = m[0];
            bool found = false;
#pragma unroll
            for (int j = 0; j < kPerThread; ++j) {
                const int cj = __popc(m[j]);
                if (!found) {
                    if (r < cj) {
                        k = j;
                        v = m[j];
                        found = true;
                    } else {
                        r -= cj;
                    }
                }
            }
            int pos = 0;
#pragma unroll
            for (int w = 16; w >= 1; w >>= 1) {
                const int c = __popc(v & ((1u << w) - 1u));
                if (r >= c) {
                    r -= c;
                    v >>= w;
                    pos += w;
                }
            }
            const int s = wbase + pos + kTileThreads * k;
            const int cz = s % TZ, col = s / TZ, cy = col % TY, cx = col / TY;
            const int x = x0 + cx, y = y0 + cy, z = z0 + cz;
            const int u = (x * Y + y) * Z + z;
            const int e = vexc[s];
            const int h = vlab[s];
            if (e <= 0 || h >= POG_INF) continue;
            const int sk = ((volatile int *)S.snk)[s];
            if (sk > 0) {
                if (h > 0) {
                    const int d = e < sk ? e : sk;
                    S.snk[s] = sk - d;
                    atomicSub(&S.exc[s], d);
                    atomicSub(g.exc + u, d);
                } else {
                    S.lab[s] = 1;
                }
                continue;
            }
            // gather: residual and far-end label of every arc, every load issued before
            // any is used
            int res[kMaxArcs], far_lab[kMaxArcs];
#pragma unroll
            for (int a = 0; a < kMaxArcs; ++a) {
                res[a] = 0;
                far_lab[a] = POG_INF;
                const int d = a >= 2 ? (a - 2) / 3 : 0;
                const int kind = a < 2 ? a : 2 + (a - 2) % 3;  // 0 down, 1 up, 2 hout, 3 hin, 4 soft
                const int dx = a < 2 ? 0 : (d == 0 ? -1 : (d == 1 ? 1 : 0));
                const int dy = a < 2 ? 0 : (d == 2 ? -1 : (d == 3 ? 1 : 0));
                const int dz = kind == 0 ? -1 : (kind == 1 ? 1 : (kind == 2 ? -D : (kind == 3 ? D : 0)));
                bool ok;
                if (kind == 0) ok = z >= 2;
                else if (kind == 1) ok = z + 1 < Z;
                else {
                    ok = (unsigned)(x + dx) < (unsigned)X && (unsigned)(y + dy) < (unsigned)Y;
                    if (kind == 2) ok = ok && z - D >= 1;
                    else if (kind == 3) ok = ok && z + D < Z;
                    else ok = ok && soft;
                }
                if (!ok) continue;
                const bool in = (unsigned)(cx + dx) < (unsigned)TX && (unsigned)(cy + dy) < (unsigned)TY &&
                                (unsigned)(cz + dz) < (unsigned)TZ;
                const int s2 = s + dz + (dy + dx * TY) * TZ;
                const int u2 = u + dz + dy * Z + dx * sx;
                if (kind == 0) res[a] = POG_CAP_INF - ((volatile int *)S.fdn)[s];
                else if (kind == 1) res[a] = in ? ((volatile int *)S.fdn)[s2] : ldcg(g.fdn + u2);
                else if (kind == 2) res[a] = POG_CAP_INF - ((volatile int *)S.fh[d])[s];
                else if (kind == 3) res[a] = in ? ((volatile int *)S.fh[d ^ 1])[s2] : ldcg(g.fh[d ^ 1] + u2);
                else if (d & 1) res[a] = g.alpha - ((volatile int *)SS.gs[d >> 1])[s];
                else res[a] = g.alpha + (in ? ((volatile int *)SS.gs[d >> 1])[s2] : ldcg(g.gs[d >> 1] + u2));
                far_lab[a] = in ? vlab[s2] : ldcg(g.lab + u2);
            }
            int best = POG_INF, bk = -1, bres = 0;
#pragma unroll
            for (int a = 0; a < kMaxArcs; ++a)
                if (res[a] > 0 && far_lab[a] < best) {
                    best = far_lab[a];
                    bk = a;
                    bres = res[a];
                }
            if (bk < 0 || h <= best) {  // relabel (Algorithm 2)
                const int nh = best >= POG_INF - 1 ? POG_INF : best + 1;
                S.lab[s] = nh;
                // the lowest residual arc found by this gather is admissible at the new
                // label (nh = its far end's label + 1): push along it in the same step
                // instead of gathering the neighbourhood again in the next local sweep
                if (nh >= POG_INF) continue;
            }
            // push along arc bk (Algorithm 2)
            const int bd = bk >= 2 ? (bk - 2) / 3 : 0;
            const int bkind = bk < 2 ? bk : 2 + (bk - 2) % 3;
            const int bdx = bk < 2 ? 0 : (bd == 0 ? -1 : (bd == 1 ? 1 : 0));
            const int bdy = bk < 2 ? 0 : (bd == 2 ? -1 : (bd == 3 ? 1 : 0));
            const int bdz = bkind == 0 ? -1 : (bkind == 1 ? 1 : (bkind == 2 ? -D : (bkind == 3 ? D : 0)));
            const int tcx = cx + bdx, tcy = cy + bdy, tcz = cz + bdz;  // target, tile-local
            const bool bin = (unsigned)tcx < (unsigned)TX && (unsigned)tcy < (unsigned)TY && (unsigned)tcz < (unsigned)TZ;
            const int bs = s + bdz + (bdy + bdx * TY) * TZ;
            const int bu = u + bdz + bdy * Z + bdx * sx;
            const int delta = e < bres ? e : bres;
            int sat = 0;
            switch (bkind) {
                case 0:
                    sat = atomicAdd(&S.fdn[s], delta) + delta == POG_CAP_INF;
                    atomicAdd(g.fdn + u, delta);
                    break;
                case 1:
                    if (bin) atomicSub(&S.fdn[bs], delta);
                    atomicSub(g.fdn + bu, delta);
                    break;
                case 2:
                    sat = atomicAdd(&S.fh[bd][s], delta) + delta == POG_CAP_INF;
                    atomicAdd(g.fh[bd] + u, delta);
                    break;
                case 3:
                    if (bin) atomicSub(&S.fh[bd ^ 1][bs], delta);
                    atomicSub(g.fh[bd ^ 1] + bu, delta);
                    break;
                default:
                    if (bd & 1) {
                        atomicAdd(&SS.gs[bd >> 1][s], delta);
                        atomicAdd(g.gs[bd >> 1] + u, delta);
                    } else {
                        if (bin) atomicSub(&SS.gs[bd >> 1][bs], delta);
                        atomicSub(g.gs[bd >> 1] + bu, delta);
                    }
                    break;
            }
            atomicSub(&S.exc[s], delta);
            atomicSub(g.exc + u, delta);
            if (bin) atomicAdd(&S.exc[bs], delta);
            // Overflow of the receiver's excess, on the global copy: checked here for large
            // pushes. A small push (below 2^20) is fire-and-forget: a tile visit brings in
            // fewer than 2^28 of them per node, so a wrap leaves the excess negative until
            // the receiver's next load (its tile is listed for the next sweep) or the next
            // global relabel, which both flag negative excess.
            if (delta >= (1 << 20)) {
                if (atomicAdd(g.exc + bu, delta) > 0x7fffffff - delta) sat = 1;
            } else {
                atomicAdd(g.exc + bu, delta);
            }
            if (sat) atomicOr(&g.ctr->error, POG_ERR_FLOW_RANGE);
            if (!bin) {  // the receiving tile has work next sweep
                if (tcz >= -TZ && tcz < 2 * TZ) {
                    const int mx = tcx < 0 ? 0 : (tcx < TX ? 1 : 2);
                    const int my = tcy < 0 ? 0 : (tcy < TY ? 1 : 2);
                    const int mz = tcz < 0 ? 0 : (tcz < TZ ? 1 : 2);
                    atomicOr(&nbmask, 1u << (mx * 9 + my * 3 + mz));
                } else {  // a vertical offset longer than a tile
                    list_tile(tile - local_tile + (((x0 + tcx) / TX) * nty + (y0 + tcy) / TY) * ntz + (z0 + tcz) / TZ,
                              L.nflag, L.nlist, L.ncount);
                }
            }
        }
    }
    __syncthreads();
    int still = 0;  // does the tile keep an active node for the next sweep?
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
        const int s = threadIdx.x + kTileThreads * k;
        bool own;
        node_of(s, own);
        still |= own && S.exc[s] > 0 && S.lab[s] < POG_INF;
    }
    const unsigned keep = __syncthreads_or(still) ? 1u << 13 : 0u;  // bit 13, (dx, dy, dz) = 0: this tile
    if (threadIdx.x < 32) {
        // warp 0 lists the tiles of the 27-bit mask: each lane claims its tile's flag, and
        // the winners take their list slots with one atomic on the sweep's shared counter
        // (one per visit instead of one per listed tile: that counter is contended)
        const int t = threadIdx.x;
        int ut = -1;
        bool won = false;
        if (t < 27 && (((nbmask | keep) >> t) & 1u)) {
            const int nx = txy / nty + t / 9 - 1, ny = txy % nty + (t / 3) % 3 - 1, nz = tz + t % 3 - 1;
            ut = tile - local_tile + (nx * nty + ny) * ntz + nz;
            won = !__ldcg(L.nflag + ut) && atomicExch(L.nflag + ut, 1) == 0;
        }
        const unsigned winners = __ballot_sync(0xffffffffu, won);
        int slot = 0;
        if (t == 0 && winners) slot = atomicAdd(L.ncount, __popc(winners));
        slot = __shfl_sync(0xffffffffu, slot, 0);
        if (won) L.nlist[slot + __popc(winners & ((1u << t) - 1u))] = ut;
    }
    if (threadIdx.x == 0) atomicAdd(&b.ctr->tiles_visited, 1ull);

    // ---- write back the owner-only words
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
        const int s = threadIdx.x + kTileThreads * k;
        bool own;
        const int u = node_of(s, own);
        if (!own) continue;
        g.lab[u] = S.lab[s];
        g.snk[u] = S.snk[s];
    }
    return true;
}

// SOFT: the shared image has room for soft arcs (some volume of the batch has alpha > 0);
// whether a given tile uses them is decided per volume. SINGLE: a batch of one volume,
// whose view comes in as a kernel parameter (read from the constant bank).
template <int TX, int TY, int TZ, bool SOFT, bool SINGLE>
__global__ void __launch_bounds__(kTileThreads, kTileBlocksPerSm) k_tile_push_relabel(Batch b, Grid g0, int tile_base0, TileLists L,
                                                                    int local_sweeps) {
    extern __shared__ int4 smem_raw[];
    // the image starts on a 128-byte boundary (bulk tensor copy destinations)
    char *img = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    TileSmem &S = *reinterpret_cast<TileSmem *>(img);
    TileSoft &SS = *reinterpret_cast<TileSoft *>(img + sizeof(TileSmem));
    __shared__ int tile_id, local_tile;
    __shared__ Grid sg;
    __shared__ unsigned nbmask;  // neighbour tiles pushed into: bit (dx+1)*9 + (dy+1)*3 + (dz+1)
    __shared__ uint64_t bar;     // completion of a visit's bulk tile copies
    unsigned phase = 0;
    const int ntiles = *L.count;
    if (blockIdx.x == 0 && threadIdx.x == 0) {  // last read by the previous sweep
        L.zero[0] = 0;
        L.zero[1] = 0;
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (SINGLE) sg = g0;  // the view in shared memory, not a local copy of the parameter
    }
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const int slot = atomicAdd(L.next, 1);
            tile_id = slot < ntiles ? L.list[slot] : -1;
            if (!SINGLE && tile_id >= 0) {
                const int vi = find_volume(b.tile_base, b.nvol, tile_id);
                sg = b.vols[vi];
                local_tile = tile_id - b.tile_base[vi];
            }
        }
        __syncthreads();
        const int tile = tile_id;
        if (tile < 0) return;
        const bool ok = tile_visit<TX, TY, TZ, SOFT>(sg, b, tile, SINGLE ? tile - tile_base0 : local_tile, L,
                                                      local_sweeps, S, SS, nbmask, &bar, phase);
        if (!ok) return;
    }
}

int sm_count() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            sms = 148;
    }
    return sms;
}

}  // namespace

// cuTensorMapEncodeTiled, looked up once through the runtime (no link against the driver
// library); null when the driver does not provide it.
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiled encode_fn() {
    static const EncodeTiled fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        return reinterpret_cast<EncodeTiled>(p);
    }();
    return fn;
}

bool encode_tile_maps(const Grid &g, int shape, void *out) {
    if (shape < 0 || shape >= kTileShapes) shape = 0;
    const EncodeTiled fn = encode_fn();
    if (!fn || g.Z % 4 != 0) return false;  // row strides must be multiples of 16 bytes
    const int *sh = kShapes[shape];
    const int32_t *arrays[kTileArrays] = {g.lab,   g.exc,   g.snk,   g.fdn,   g.fh[0],
                                          g.fh[1], g.fh[2], g.fh[3], g.gs[0], g.gs[1]};
    const int narr = g.gs[0] ? kTileArrays : kTileArrays - 2;
    const cuuint64_t dims[3] = {(cuuint64_t)g.Z, (cuuint64_t)g.Y, (cuuint64_t)g.X};
    const cuuint64_t strides[2] = {(cuuint64_t)g.Z * 4, (cuuint64_t)g.Y * g.Z * 4};
    const cuuint32_t box[3] = {(cuuint32_t)sh[2], (cuuint32_t)sh[1], (cuuint32_t)sh[0]};
    const cuuint32_t unit[3] = {1, 1, 1};
    static_assert(sizeof(CUtensorMap) == kTensorMapBytes, "tensor map size");
    for (int a = 0; a < narr; ++a) {
        if (reinterpret_cast<uintptr_t>(arrays[a]) % 16 != 0) return false;
        CUtensorMap m;
        if (fn(&m, CU_TENSOR_MAP_DATA_TYPE_INT32, 3, const_cast<int32_t *>(arrays[a]), dims, strides, box, unit,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
        std::memcpy(static_cast<char *>(out) + a * kTensorMapBytes, &m, kTensorMapBytes);
    }
    return true;
}

long long tile_count(const Grid &g, int shape) {
    const TileGeom t = geom(g, shape < 0 || shape >= kTileShapes ? 0 : shape);
    return (long long)t.ntx * t.nty * t.ntz;
}

long long tile_count_max(const Grid &g) {
    long long m = 0;
    for (int i = 0; i < kTileShapes; ++i) m = tile_count(g, i) > m ? tile_count(g, i) : m;
    return m;
}

template <int TX, int TY, int TZ, bool SOFT, bool SINGLE>
cudaError_t launch_tile_instance(const Batch &b, const Grid &g0, int tile_base0, const TileLists &L, int local_sweeps,
                                 int blocks, cudaStream_t st) {
    const size_t smem = sizeof(TileSmem) + (SOFT ? sizeof(TileSoft) : 0) + 128;  // + alignment slack
    static bool configured = false;
    if (!configured) {
        const cudaError_t e = cudaFuncSetAttribute(k_tile_push_relabel<TX, TY, TZ, SOFT, SINGLE>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    k_tile_push_relabel<TX, TY, TZ, SOFT, SINGLE><<<blocks, kTileThreads, smem, st>>>(b, g0, tile_base0, L,
                                                                                      local_sweeps);
    return cudaGetLastError();
}

template <int TX, int TY, int TZ>
cudaError_t launch_tile_kernel(const Batch &b, const Grid *single, int single_tile_base, bool soft,
                               const TileLists &L, int local_sweeps, int blocks, cudaStream_t st) {
    const Grid g0 = single ? *single : Grid{};
    const int t0 = single_tile_base;
    if (single)
        return soft ? launch_tile_instance<TX, TY, TZ, true, true>(b, g0, t0, L, local_sweeps, blocks, st)
                    : launch_tile_instance<TX, TY, TZ, false, true>(b, g0, t0, L, local_sweeps, blocks, st);
    return soft ? launch_tile_instance<TX, TY, TZ, true, false>(b, g0, 0, L, local_sweeps, blocks, st)
                : launch_tile_instance<TX, TY, TZ, false, false>(b, g0, 0, L, local_sweeps, blocks, st);
}

// The tile lists of sweep k alternate between two buffers, k mod 2: buffer k's tiles are
// visited, and visits list the next sweep's tiles in the other buffer (whose flags are
// all clear: every visit clears its own flag). Their counters rotate through three
// pairs, k mod 3: sweep k reads pair k, appends through pair k+1, and zeroes pair k+2
// (last read by sweep k-1), so a sweep is one launch. After a global relabel, activity
// is recomputed and volumes may have left the batch, so the first sweep of a round
// (`full_scan`) drops its carried list and scans every node of the batch into it.
// `tiles` holds [flag p][list p] for p = 0, 1 (4 arrays of `ntiles`); `work` 3 pairs
// of ints, all zero before sweep 0. `soft`: some volume has alpha > 0; `single`: the view
// of the only volume (whose tiles start at union tile `single_tile_base`), or null.
cudaError_t launch_tile_sweep(const Batch &b, const Grid *single, int single_tile_base, bool soft, int shape,
                              int *tiles, long long ntiles, int *work, long long serial, bool full_scan,
                              int local_sweeps, cudaStream_t st) {
    if (shape < 0 || shape >= kTileShapes) shape = 0;
    const int p = (int)(serial & 1), q = p ^ 1;
    int *flag[2] = {tiles, tiles + 2 * ntiles};
    int *list[2] = {tiles + ntiles, tiles + 3 * ntiles};
    int *cnt = work + 2 * (int)(serial % 3);
    int *ncnt = work + 2 * (int)((serial + 1) % 3);
    int *zcnt = work + 2 * (int)((serial + 2) % 3);
    const int sms = sm_count();
    const int *sh = kShapes[shape];
    if (full_scan) {
        k_clear_listed<<<sms, 256, 0, st>>>(flag[p], list[p], cnt);
        const cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int), st);
        if (e != cudaSuccess) return e;
        k_collect_tiles<<<sms * 8, 256, 0, st>>>(b, sh[0], sh[1], sh[2], flag[p], list[p], cnt);
    }
    TileLists L{list[p], cnt, flag[p], cnt + 1, list[q], ncnt, flag[q], zcnt};
    const int blocks = sms * kTileBlocksPerSm;
    switch (shape) {
        case 1: return launch_tile_kernel<8, 8, 16>(b, single, single_tile_base, soft, L, local_sweeps, blocks, st);
        case 2: return launch_tile_kernel<4, 4, 64>(b, single, single_tile_base, soft, L, local_sweeps, blocks, st);
        case 3: return launch_tile_kernel<2, 4, 128>(b, single, single_tile_base, soft, L, local_sweeps, blocks, st);
        default: return launch_tile_kernel<4, 8, 32>(b, single, single_tile_base, soft, L, local_sweeps, blocks, st);
    }
}

}  // namespace pog
