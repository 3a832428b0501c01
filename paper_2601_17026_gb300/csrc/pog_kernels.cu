// Node-parallel kernels of the GB300 min-cut solver: graph construction, push/relabel
// sweeps, global relabelling by reverse BFS, gap relabelling, termination counts, cut
// extraction, surface heights, quantisation and the energy backward.
#include <cooperative_groups.h>

#include "pog_internal.cuh"
#include "pog_launch.h"

namespace pog {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of a 64-bit value, added once per block into *dst.
__device__ __forceinline__ void block_add_u64(unsigned long long v, unsigned long long *dst) {
    __shared__ unsigned long long part[kThreads / 32];
    v = warp_sum_u64(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) part[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < (int)(blockDim.x >> 5) ? part[lane] : 0ull;
        v = warp_sum_u64(v);
        if (lane == 0 && v != 0ull) atomicAdd(dst, v);
    }
}

inline int blocks_for(long long n) { return (int)((n + kThreads - 1) / kThreads); }

// ----------------------------------------------------------------------------------
// Graph construction (Section 1.2): node weights w(z) = c(z) - c(z-1) become source
// excess (w < 0) or sink residual (w > 0); arcs start empty; labels start at 0.
// ----------------------------------------------------------------------------------

struct CostI32 {
    const int32_t *c;
    __device__ __forceinline__ int load(int i, int &err) const {
        const int v = c[i];
        if (v >= (1 << 30) || v <= -(1 << 30)) err |= POG_ERR_COST_RANGE;
        return v;
    }
};

struct CostF32 {
    const float *c;
    float scale;
    const int32_t *h_aug;  // optional surface whose nodes get `margin` added
    int margin;
    int Z;
    __device__ __forceinline__ int load(int i, int &err) const {
        const float v = c[i] * scale;  // exact for a power-of-two scale
        if (!(fabsf(v) < 1073741824.0f)) {  // also rejects NaN / Inf
            err |= POG_ERR_COST_RANGE;
            return 0;
        }
        int q = __float2int_rn(v);  // round half to even
        if (h_aug && h_aug[i / Z] == i % Z) q += margin;
        return q;
    }
};

template <class Cost>
__global__ void k_build(Grid g, Cost cost) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long src = 0, bsum = 0, bpos = 0, bneg = 0;
    int err = 0;
    if (u < g.N) {
        const int z = u % g.Z;
        const int c = cost.load(u, err);
        int e = 0, s = 0, l = POG_INF;
        if (z == 0) {
            bsum = (unsigned long long)(long long)c;
            if (u != 0 && c > 0) bpos = (unsigned long long)c;
            if (u != 0 && c < 0) bneg = (unsigned long long)(-(long long)c);
        } else {
            const int w = c - cost.load(u - 1, err);
            e = w < 0 ? -w : 0;
            s = w > 0 ? w : 0;
            l = 0;
            src = (unsigned long long)e;
        }
        g.lab[u] = l;
        g.exc[u] = e;
        g.snk[u] = s;
        g.fdn[u] = 0;
#pragma unroll
        for (int d = 0; d < 4; ++d) g.fh[d][u] = 0;
        if (g.gs[0]) {
            g.gs[0][u] = 0;
            g.gs[1][u] = 0;
        }
    }
    if (err) atomicOr(&g.ctr->error, err);
    block_add_u64(src, &g.ctr->src_total);
    __syncthreads();
    block_add_u64(bsum, &g.ctr->bottom_sum);
    __syncthreads();
    block_add_u64(bpos, &g.ctr->pos_bottom);
    __syncthreads();
    block_add_u64(bneg, &g.ctr->neg_part);
}

// The bottom node of column (0,0) carries the offset -(1 + sum c(., ., 0)); the bottom
// layer's sink arcs give a constant part of the flow value.
template <class Cost>
__global__ void k_bottom_const(Grid g, Cost cost) {
    int err = 0;
    const long long c00 = cost.load(0, err);
    const long long w00 = c00 - 1 - (long long)g.ctr->bottom_sum;
    g.ctr->bottom_const = g.ctr->pos_bottom + (unsigned long long)(w00 > 0 ? w00 : 0);
    g.ctr->neg_bottom = g.ctr->neg_part + (unsigned long long)(w00 < 0 ? -w00 : 0);
}

// ----------------------------------------------------------------------------------
// Warm start of the loss-augmented problem (structured hinge): the costs change only at
// node (x, y, t) of every column, t = h_t(x, y), by +margin. So w(t) grows by margin and
// w(t+1) shrinks by margin, and the final residual state of the plain problem becomes a
// valid preflow of the augmented one by two capacity increases per column: the sink arc
// of (x, y, t) gains margin (its residual grows), and node (x, y, t+1) gains a source arc
// of capacity margin, saturated at once (its excess grows). Its terminal capacities are
// then cs = max(-w, 0) + margin, ct = max(w, 0) (and at t: cs = max(-w, 0), ct = max(w, 0) +
// margin), i.e. min(cs, ct) may exceed 0; every s-t cut then has capacity larger by
// sum min(cs, ct) than in the graph with cs = max(-w', 0), ct = max(w', 0), so the cut is
// the same and the max-flow value of that graph is the one found minus `aug_offset`. When
// t = 0 the bottom layer's weights change, whose constants are recomputed from the
// augmented costs (k_bottom_sums, k_bottom_const). The source supply of the nodes above
// the bottom layer (src_total) grows by margin per node t+1.
// ----------------------------------------------------------------------------------

// Bottom-layer sums of k_build alone (one thread per column), on possibly augmented costs.
template <class Cost>
__global__ void k_bottom_sums(Grid g, Cost cost) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long bsum = 0, bpos = 0, bneg = 0;
    int err = 0;
    if (col < g.X * g.Y) {
        const int u = col * g.Z;
        const int c = cost.load(u, err);
        bsum = (unsigned long long)(long long)c;
        if (u != 0 && c > 0) bpos = (unsigned long long)c;
        if (u != 0 && c < 0) bneg = (unsigned long long)(-(long long)c);
    }
    if (err) atomicOr(&g.ctr->error, err);
    block_add_u64(bsum, &g.ctr->bottom_sum);
    __syncthreads();
    block_add_u64(bpos, &g.ctr->pos_bottom);
    __syncthreads();
    block_add_u64(bneg, &g.ctr->neg_part);
}

// One thread per column: the capacity increases at t and t+1 (plain costs give w).
__global__ void k_augment(Grid g, CostF32 plain, const int32_t *ht, int margin) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long supply = 0, offset = 0;
    int err = 0;
    if (col < g.X * g.Y) {
        const int t = ht[col];
        const int base = col * g.Z;
        if (t >= 1 && t < g.Z) {
            const int w = plain.load(base + t, err) - plain.load(base + t - 1, err);
            const long long r = (long long)g.snk[base + t] + margin;
            if (r > 0x7fffffffll) err |= POG_ERR_FLOW_RANGE;
            g.snk[base + t] = (int)r;
            if (w < 0) offset += (unsigned long long)min(-w, margin);
        }
        if (t >= 0 && t + 1 < g.Z) {
            const int w = plain.load(base + t + 1, err) - plain.load(base + t, err);
            const long long e = (long long)g.exc[base + t + 1] + margin;
            if (e > 0x7fffffffll) err |= POG_ERR_FLOW_RANGE;
            g.exc[base + t + 1] = (int)e;
            supply += (unsigned long long)margin;
            if (w > 0) offset += (unsigned long long)min(w, margin);
        }
        if (t < 0 || t >= g.Z) err |= POG_ERR_COST_RANGE;  // not a surface
    }
    if (err) atomicOr(&g.ctr->error, err);
    block_add_u64(supply, &g.ctr->src_total);
    __syncthreads();
    block_add_u64(offset, &g.ctr->aug_offset);
}

// ----------------------------------------------------------------------------------
// Column pre-push: before the first global relabel, every column pushes its excess down
// its infinite down arcs (Section 1.2: (x,y,z) -> (x,y,z-1)), absorbing it into the sink
// arcs it passes. Scanning from the top, the flow leaving node z downwards is
//   c_z = max(0, c_{z+1} + e_z - s_z),
// a composition of maps c -> max(b, c + a) that a warp evaluates as a prefix scan over 32
// heights at a time. What reaches z = 1 stays there as excess. Only pushes along
// residual arcs are made, so the result is a preflow; it is the starting point of
// push-relabel (the paper starts from the saturated source arcs alone).
// ----------------------------------------------------------------------------------

__global__ void k_column_prepush(Grid g) {
    const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (col >= g.X * g.Y) return;
    const long long base = (long long)col * g.Z;
    long long carry = 0;  // flow entering the current chunk from above
    bool overflow = false;
    for (int zhi = g.Z - 1; zhi >= 1; zhi -= 32) {
        const int z = zhi - lane;  // lane 0 is the top of the chunk
        const bool valid = z >= 1;
        const long long e = valid ? g.exc[base + z] : 0;
        const long long sk = valid ? g.snk[base + z] : 0;
        long long a = e - sk, b = 0;  // this node's map c -> max(b, c + a)
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {  // compose with the maps of the nodes above
            const long long pa = __shfl_up_sync(0xffffffffu, a, off);
            const long long pb = __shfl_up_sync(0xffffffffu, b, off);
            if (lane >= off) {
                b = max(b, pb + a);
                a = pa + a;
            }
        }
        const long long c_out = max(b, carry + a);
        long long c_in = __shfl_up_sync(0xffffffffu, c_out, 1);
        if (lane == 0) c_in = carry;
        if (valid) {
            const long long absorbed = c_in + e - c_out;  // into the sink arc
            g.snk[base + z] = (int)(sk - absorbed);
            if (z >= 2) {
                const long long f = (long long)g.fdn[base + z] + c_out;  // adds to any flow already there
                g.fdn[base + z] = (int)f;
                g.exc[base + z] = 0;
                if (f >= 0x7fffffffll) overflow = true;
            } else {
                g.exc[base + z] = (int)c_out;
            }
            if (c_out > 0x7fffffffll) overflow = true;
        }
        carry = __shfl_sync(0xffffffffu, c_out, 31);
    }
    if (overflow) atomicOr(&g.ctr->error, POG_ERR_FLOW_RANGE);
}

// ----------------------------------------------------------------------------------
// Push/relabel sweep (Section 2.1, Algorithm 2), lock-free: each node is discharged
// only by its own thread; neighbours' excess and the paired arc values are changed
// with atomics. Every value a thread reads can only move, concurrently, in the
// direction that makes its push smaller than allowed, so stale reads are safe.
// ----------------------------------------------------------------------------------

// Arc kind of a gathered slot (see gather_out).
__device__ __forceinline__ int slot_kind(int k) {
    if (k == 0) return ARC_DOWN;
    if (k == 1) return ARC_UP;
    const int r = (k - 2) % 3;
    return r == 0 ? ARC_HOUT : (r == 1 ? ARC_HIN : ARC_SOFT);
}

template <bool SOFT>
__device__ __forceinline__ void discharge(const Grid &g, int u, int ops) {
    const int z = u % g.Z;
    if (z == 0) return;
    const int col = u / g.Z;
    const int x = col / g.Y, y = col - x * g.Y;
    for (int it = 0; it < ops; ++it) {
        const int e = ldcg(g.exc + u);
        const int h = ldcg(g.lab + u);
        if (e <= 0 || h >= POG_INF) return;
        const int s = ldcg(g.snk + u);
        if (s > 0) {  // the sink arc: label 0, always the lowest
            if (h > 0) {
                const int delta = e < s ? e : s;
                g.snk[u] = s - delta;
                atomicSub(g.exc + u, delta);
            } else {
                g.lab[u] = 1;
            }
            continue;
        }
        Hood hd;
        gather_out<SOFT>(g, u, x, y, z, hd);
        int best = POG_INF, k = -1;
#pragma unroll
        for (int i = 0; i < kMaxArcs; ++i)
            if (hd.lab[i] < best) {
                best = hd.lab[i];
                k = i;
            }
        if (k < 0 || h <= best) {  // relabel (Algorithm 2): one above the lowest residual neighbour
            g.lab[u] = best >= POG_INF - 1 ? POG_INF : best + 1;
            continue;
        }
        int res = 0, target = 0;
#pragma unroll
        for (int i = 0; i < kMaxArcs; ++i)
            if (i == k) {
                res = hd.res[i];
                target = hd.node[i];
            }
        const int delta = e < res ? e : res;
        const int kind = slot_kind(k);
        const int dir = k >= 2 ? (k - 2) / 3 : 0;
        int sat = 0;
        switch (kind) {
            case ARC_DOWN: sat = atomicAdd(g.fdn + u, delta) + delta == POG_CAP_INF; break;
            case ARC_UP: atomicSub(g.fdn + u + 1, delta); break;
            case ARC_HOUT: sat = atomicAdd(g.fh[dir] + u, delta) + delta == POG_CAP_INF; break;
            case ARC_HIN: atomicSub(g.fh[dir ^ 1] + target, delta); break;
            default:
                if (dir & 1) atomicAdd(g.gs[dir >> 1] + u, delta);
                else atomicSub(g.gs[dir >> 1] + target, delta);
                break;
        }
        atomicSub(g.exc + u, delta);
        const int old = atomicAdd(g.exc + target, delta);
        if (old > 0x7fffffff - delta) sat = 1;
        if (sat) atomicOr(&g.ctr->error, POG_ERR_FLOW_RANGE);
    }
}

// A sweep is two launches: the active nodes (excess > 0, finite label) are compacted
// into a list by a coalesced scan, then one thread per listed node discharges it with
// up to `ops` push or relabel operations. Clustered active nodes thus spread over all
// threads instead of serialising on the few that own their region.
__global__ void __launch_bounds__(kThreads) k_collect_active(Batch b, int *list, int *count) {
    const int stride = gridDim.x * blockDim.x;
    for (int vi = 0; vi < b.nvol; ++vi) {
        const Grid g = b.vols[vi];
        const int base = b.node_base[vi];
        for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < g.N; u += stride) {
            if (__ldcg(g.exc + u) <= 0 || u % g.Z == 0 || __ldcg(g.lab + u) >= POG_INF) continue;
            namespace cg = cooperative_groups;
            const cg::coalesced_group grp = cg::coalesced_threads();
            int at = 0;
            if (grp.thread_rank() == 0) at = atomicAdd(count, (int)grp.size());
            at = grp.shfl(at, 0);
            list[at + grp.thread_rank()] = base + u;
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_push_relabel(Batch b, const int *list, const int *count, int ops) {
    const int n = *count;
    const int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int uv = list[i];
        const int vi = find_volume(b.node_base, b.nvol, uv);
        const Grid g = b.vols[vi];
        const int u = uv - b.node_base[vi];
        if (g.gs[0]) discharge<true>(g, u, ops);
        else discharge<false>(g, u, ops);
    }
}

// ----------------------------------------------------------------------------------
// Gap relabelling (Section 2.1): if no node has label g while some have g < d < INF,
// those cannot reach t and are raised to INF. Level occupancy is a bitmap.
// ----------------------------------------------------------------------------------

constexpr int kGapSharedWords = 256;  // levels below 8192 are gathered per block first

__global__ void k_gap_occupancy(Batch b, unsigned int *bits, int levels) {
    __shared__ unsigned int local[kGapSharedWords];
    for (int i = threadIdx.x; i < kGapSharedWords; i += blockDim.x) local[i] = 0u;
    __syncthreads();
    const int stride = gridDim.x * blockDim.x;
    int lmax = 0;
    for (int vi = 0; vi < b.nvol; ++vi) {
        const Grid g = b.vols[vi];
        for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < g.N; u += stride) {
            if (u % g.Z == 0) continue;
            const int l = g.lab[u];
            if (l < kGapSharedWords * 32) atomicOr(local + (l >> 5), 1u << (l & 31));
            else if (l < levels) atomicOr(bits + (l >> 5), 1u << (l & 31));
            if (l < POG_INF && l > lmax) lmax = l;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lmax = max(lmax, __shfl_down_sync(0xffffffffu, lmax, o));
    if ((threadIdx.x & 31) == 0 && lmax > 0) atomicMax(&b.ctr->max_label, lmax);
    __syncthreads();
    for (int i = threadIdx.x; i < kGapSharedWords; i += blockDim.x)
        if (local[i]) atomicOr(bits + i, local[i]);
}

// One block: the first empty level above 0 that lies below the largest finite label.
__global__ void k_gap_find(Batch b, const unsigned int *bits, int levels) {
    __shared__ int first;
    if (threadIdx.x == 0) first = 0x7fffffff;
    __syncthreads();
    const int lmax = min(b.ctr->max_label, levels - 1);
    for (int w = threadIdx.x; w * 32 <= lmax; w += blockDim.x) {
        unsigned int empty = ~bits[w];
        if (w == 0) empty &= ~1u;  // level 0 is the sink itself
        if (empty) {
            const int l = w * 32 + __ffs(empty) - 1;
            if (l < lmax) atomicMin(&first, l);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) b.ctr->gap_level = first == 0x7fffffff ? 0 : first;
}

__global__ void k_gap_raise(Batch b) {
    const int gap = b.ctr->gap_level;
    const int stride = gridDim.x * blockDim.x;
    unsigned long long r = 0;
    if (gap > 0) {
        for (int vi = 0; vi < b.nvol; ++vi) {
            const Grid g = b.vols[vi];
            for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < g.N; u += stride) {
                if (u % g.Z == 0) continue;
                const int l = g.lab[u];
                if (l > gap && l < POG_INF) {
                    g.lab[u] = POG_INF;
                    ++r;
                }
            }
        }
    }
    block_add_u64(r, &b.ctr->raised);
}

// One warp per column: the top marked node (0 when only the bottom layer is in S).
__global__ void k_heights(Grid g, int32_t *heights) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int cols = g.X * g.Y;
    if (warp >= cols) return;
    const int32_t *m = g.lab + (long long)warp * g.Z;
    int top = 0;
    for (int z0 = 0; z0 < g.Z; z0 += 32) {
        const int z = z0 + lane;
        const unsigned b = __ballot_sync(0xffffffffu, z >= 1 && z < g.Z && m[z] != 0);
        if (b) top = z0 + 31 - __clz(b);
    }
    if (lane == 0) heights[warp] = top;
}

__global__ void k_excess_sum(Grid g) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long e = 0;
    if (u < g.N && u % g.Z != 0) e = (unsigned long long)(long long)g.exc[u];
    block_add_u64(e, &g.ctr->excess_sum);
}

// ----------------------------------------------------------------------------------
// Quantisation and the energy backward.
// ----------------------------------------------------------------------------------

__global__ void k_quantise(const float *in, int32_t *out, long long n, float scale, int *err) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float v = in[i] * scale;
    if (!(fabsf(v) < 1073741824.0f)) {
        atomicOr(err, POG_ERR_COST_RANGE);
        out[i] = 0;
        return;
    }
    out[i] = __float2int_rn(v);
}

// grad = g_e * onehot(h) + g_h * (onehot(h_target) - onehot(h_hat)); each thread writes
// four consecutive z of one column (vectorised when Z is a multiple of 4).
__global__ void k_backward(float *grad, const int32_t *h, const int32_t *ht, const int32_t *hh,
                           const float *ge, const float *gh, int B, int XY, int Z) {
    const long long n = (long long)B * XY * Z;
    const long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (i >= n) return;
    for (int k = 0; k < 4 && i + k < n; ++k) {
        const long long e = i + k;
        const long long colg = e / Z;  // b * XY + col
        const int z = (int)(e - colg * Z);
        const int b = (int)(colg / XY);
        float v = (h[colg] == z) ? ge[b] : 0.0f;
        if (gh) {
            const float s = gh[b];
            if (ht[colg] == z) v += s;
            if (hh[colg] == z) v -= s;
        }
        grad[e] = v;
    }
}

// Surface energy of Eq. 1 on the quantised costs, one block per volume:
// sum_col cq(col, h) + alpha * sum over unordered 4-neighbour pairs |h_p - h_q|.
__global__ void k_surface_energy(const float *cost, float scale, const int32_t *h, int X, int Y, int Z, int alpha,
                                 long long *out) {
    const int b = blockIdx.x;
    const int XY = X * Y;
    const float *c = cost + (long long)b * XY * Z;
    const int32_t *hb = h + (long long)b * XY;
    unsigned long long acc = 0;
    int bad = 0;
    for (int col = threadIdx.x; col < XY; col += blockDim.x) {
        const int x = col / Y, y = col - x * Y;
        const int hp = hb[col];
        if (hp < 0 || hp >= Z) {  // not a surface: reported as INT64_MIN
            bad = 1;
            continue;
        }
        long long e = __float2int_rn(c[(long long)col * Z + hp] * scale);
        if (x + 1 < X) e += (long long)alpha * abs(hp - hb[col + Y]);
        if (y + 1 < Y) e += (long long)alpha * abs(hp - hb[col + 1]);
        acc += (unsigned long long)e;
    }
    __shared__ unsigned long long part[kThreads / 32];
    __shared__ int any_bad;
    if (threadIdx.x == 0) any_bad = 0;
    __syncthreads();
    if (bad) any_bad = 1;
    acc = warp_sum_u64(acc);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        out[b] = any_bad ? (long long)0x8000000000000000ull : (long long)t;
    }
}

}  // namespace

// ---------------------------------------------------------------------------------- launchers

#define POG_LAUNCH(kernel, n, stream, ...)                                          \
    do {                                                                            \
        kernel<<<blocks_for(n), kThreads, 0, stream>>>(__VA_ARGS__);                \
        return cudaGetLastError();                                                  \
    } while (0)

cudaError_t launch_build_i32(const Grid &g, const int32_t *cost, cudaStream_t st) {
    CostI32 c{cost};
    k_build<<<blocks_for(g.N), kThreads, 0, st>>>(g, c);
    k_bottom_const<<<1, 1, 0, st>>>(g, c);
    return cudaGetLastError();
}

cudaError_t launch_build_f32(const Grid &g, const float *cost, float scale, const int32_t *h_aug, int margin,
                             cudaStream_t st) {
    CostF32 c{cost, scale, h_aug, margin, g.Z};
    k_build<<<blocks_for(g.N), kThreads, 0, st>>>(g, c);
    k_bottom_const<<<1, 1, 0, st>>>(g, c);
    return cudaGetLastError();
}

cudaError_t launch_augment(const Grid &g, const float *cost, float scale, const int32_t *ht, int margin,
                           cudaStream_t st) {
    // the five bottom-layer sums are consecutive counters: clear them, then recompute
    cudaError_t e = cudaMemsetAsync(&g.ctr->bottom_sum, 0, 5 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(&g.ctr->aug_offset, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
    const CostF32 aug{cost, scale, ht, margin, g.Z};
    const CostF32 plain{cost, scale, nullptr, 0, g.Z};
    const long long cols = (long long)g.X * g.Y;
    k_bottom_sums<<<blocks_for(cols), kThreads, 0, st>>>(g, aug);
    k_bottom_const<<<1, 1, 0, st>>>(g, aug);
    k_augment<<<blocks_for(cols), kThreads, 0, st>>>(g, plain, ht, margin);
    return cudaGetLastError();
}

cudaError_t launch_column_prepush(const Grid &g, cudaStream_t st) {
    const long long threads = (long long)g.X * g.Y * 32;
    POG_LAUNCH(k_column_prepush, threads, st, g);
}

int grid_blocks() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            sms = 148;
    }
    return sms * 8;
}

cudaError_t launch_sweep(const Batch &b, int *list, int *count, int ops, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    const int blocks = grid_blocks();
    k_collect_active<<<blocks, kThreads, 0, st>>>(b, list, count);
    k_push_relabel<<<blocks, kThreads, 0, st>>>(b, list, count, ops);
    return cudaGetLastError();
}

cudaError_t launch_gap(const Batch &b, unsigned int *bits, int levels, cudaStream_t st) {
    const cudaError_t e = cudaMemsetAsync(bits, 0, (size_t)(levels / 32) * sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    const int blocks = grid_blocks();
    k_gap_occupancy<<<blocks, kThreads, 0, st>>>(b, bits, levels);
    k_gap_find<<<1, 1024, 0, st>>>(b, bits, levels);
    k_gap_raise<<<blocks, kThreads, 0, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_heights(const Grid &g, int32_t *heights, cudaStream_t st) {
    const long long threads = (long long)g.X * g.Y * 32;
    POG_LAUNCH(k_heights, threads, st, g, heights);
}

cudaError_t launch_excess_sum(const Grid &g, cudaStream_t st) { POG_LAUNCH(k_excess_sum, g.N, st, g); }

cudaError_t launch_quantise(const float *in, int32_t *out, long long n, float scale, int *err, cudaStream_t st) {
    POG_LAUNCH(k_quantise, n, st, in, out, n, scale, err);
}

cudaError_t launch_backward(float *grad, const int32_t *h, const int32_t *ht, const int32_t *hh, const float *ge,
                            const float *gh, int B, int XY, int Z, cudaStream_t st) {
    const long long n = ((long long)B * XY * Z + 3) / 4;
    POG_LAUNCH(k_backward, n, st, grad, h, ht, hh, ge, gh, B, XY, Z);
}

cudaError_t launch_surface_energy(const float *cost, float scale, const int32_t *h, int B, int X, int Y, int Z,
                                  int alpha, long long *out, cudaStream_t st) {
    k_surface_energy<<<B, kThreads, 0, st>>>(cost, scale, h, X, Y, Z, alpha, out);
    return cudaGetLastError();
}

}  // namespace pog
