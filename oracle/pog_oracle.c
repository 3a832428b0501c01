/*
 * CPU oracle for the proper-order multi-column min-cut. TEST INFRASTRUCTURE ONLY:
 * only the tests, the smoke check and the CPU-baseline leg of the benchmark may call
 * it. It shares no code with the CUDA path.
 *
 * What it computes (plain and slow on purpose):
 *   1. The literal s-t graph of the optimal net-surface problem (Section 1.2): every
 *      node weight w(v) becomes a terminal arc, every proper-order edge becomes an
 *      explicit arc with an explicit reverse half-arc. Nothing is contracted or
 *      dropped; the edge list is stored, the opposite of the implicit addressing of
 *      Section 3.2.3.
 *   2. Dinic's blocking-flow max-flow (Section 2), int64 capacities.
 *   3. The minimal minimum cut: the nodes reachable from s in the final residual
 *      graph, and from it the surface height of each column.
 *   4. The surface energy of Eq. 1 and the cut capacity of Eq. 6, from their
 *      definitions, for the identities that pin the oracle.
 *
 * Graph (z fastest: node (x,y,z) has index (x*Y + y)*Z + z; s = N, t = N+1):
 *   w(x,y,z) = c(x,y,z) - c(x,y,z-1) for z > 0, w(x,y,0) = c(x,y,0), and
 *   w(0,0,0) is further lowered by 1 + sum_{x,y} c(x,y,0) so the cut is never empty.
 *   s -> v with capacity -w(v) when w(v) < 0; v -> t with capacity w(v) when w(v) > 0.
 *   (x,y,z) -> (x,y,z-1), infinite, for z >= 1            (column order)
 *   (x,y,z) -> (x',y',max(0,z-delta)), infinite            (hard smoothness, each
 *                                                           in-grid 4-neighbour)
 *   (x,y,z) -> (x',y',z), capacity alpha, if alpha > 0     (soft smoothness: one arc
 *                                                           per ordered neighbour pair)
 *
 * General convex pairwise cost (the convex edge costs of an edge interval, Section 1.2):
 * E_prior = sum over unordered 4-neighbour pairs of f(|h_p - h_q|), f(0) = 0, f convex
 * on 0..delta. It is the sum of layers d = 0..delta-1 of soft arcs
 *   (x,y,z) -> (x',y',z-d), capacity k_d, for z - d >= 0,
 * with k_0 = f(1) and k_d = f(d+1) - 2 f(d) + f(d-1) (the second difference of f): the
 * layer-d arcs from column p to column q that a surface cuts are those with
 * h_q + d < z <= h_p, (h_p - h_q - d)^+ of them, and sum_d k_d (t - d)^+ = f(t) for
 * 0 <= t <= delta. The linear penalty alpha |h_p - h_q| is the single layer k_0 = alpha.
 * An arc whose head would lie below z = 0 is never cut (that node is in every closed
 * set) and is left out.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_INF ((int64_t)1 << 62)

enum { ORC_OK = 0, ORC_E_ARGS = 1, ORC_E_NOMEM = 2, ORC_E_CAPACITY = 3,
       ORC_E_CONSERVATION = 4, ORC_E_CUT = 5, ORC_E_SURFACE = 6 };

typedef struct {
    int64_t n;        /* nodes including s and t */
    int64_t m;        /* half-arcs */
    int64_t *first;   /* CSR row starts, n+1 entries */
    int32_t *head;    /* head node of each half-arc */
    int64_t *rev;     /* index of the paired half-arc */
    int64_t *cap;     /* residual capacity */
    int64_t *cap0;    /* initial capacity (only when invariants are checked) */
    int64_t *fill;    /* scratch: next free slot per node during construction */
} orc_graph;

static int64_t idx3(int32_t Y, int32_t Z, int64_t x, int64_t y, int64_t z) {
    return (x * Y + y) * Z + z;
}

/* Node weight of Section 1.2 (the bottom node of column (0,0) carries the offset). */
static int64_t node_weight(const int32_t *c, int32_t X, int32_t Y, int32_t Z,
                           int64_t x, int64_t y, int64_t z, int64_t bottom_sum) {
    (void)X;
    int64_t w = (z > 0) ? (int64_t)c[idx3(Y, Z, x, y, z)] - (int64_t)c[idx3(Y, Z, x, y, z - 1)]
                        : (int64_t)c[idx3(Y, Z, x, y, 0)];
    if (x == 0 && y == 0 && z == 0) w -= 1 + bottom_sum;
    return w;
}

static int64_t bottom_layer_sum(const int32_t *c, int32_t X, int32_t Y, int32_t Z) {
    int64_t s = 0;
    for (int64_t x = 0; x < X; ++x)
        for (int64_t y = 0; y < Y; ++y) s += c[idx3(Y, Z, x, y, 0)];
    return s;
}

static const int DX[4] = {-1, 1, 0, 0};
static const int DY[4] = {0, 0, -1, 1};

/* Visit every arc of the literal graph once. mode 0 counts half-arcs per node,
 * mode 1 places them. */
static void add_arc(orc_graph *g, int mode, int64_t u, int64_t v, int64_t c) {
    if (mode == 0) {
        g->first[u + 1]++;
        g->first[v + 1]++;
        return;
    }
    int64_t a = g->fill[u]++;
    int64_t b = g->fill[v]++;
    g->head[a] = (int32_t)v;
    g->head[b] = (int32_t)u;
    g->rev[a] = b;
    g->rev[b] = a;
    g->cap[a] = c;
    g->cap[b] = 0;
    if (g->cap0) {
        g->cap0[a] = c;
        g->cap0[b] = 0;
    }
}

/* Soft layers: kcap[d] is the capacity of the arcs that drop d heights, d < nk. */
static void enumerate_arcs(orc_graph *g, int mode, const int32_t *c, int32_t X, int32_t Y,
                           int32_t Z, int32_t delta, const int64_t *kcap, int32_t nk) {
    const int64_t N = (int64_t)X * Y * Z, s = N, t = N + 1;
    const int64_t bsum = bottom_layer_sum(c, X, Y, Z);
    for (int64_t x = 0; x < X; ++x)
        for (int64_t y = 0; y < Y; ++y)
            for (int64_t z = 0; z < Z; ++z) {
                const int64_t v = idx3(Y, Z, x, y, z);
                const int64_t w = node_weight(c, X, Y, Z, x, y, z, bsum);
                if (w < 0) add_arc(g, mode, s, v, -w);
                if (w > 0) add_arc(g, mode, v, t, w);
                if (z >= 1) add_arc(g, mode, v, idx3(Y, Z, x, y, z - 1), ORC_INF);
                for (int d = 0; d < 4; ++d) {
                    const int64_t xq = x + DX[d], yq = y + DY[d];
                    if (xq < 0 || xq >= X || yq < 0 || yq >= Y) continue;
                    const int64_t zq = (z - delta > 0) ? z - delta : 0;
                    add_arc(g, mode, v, idx3(Y, Z, xq, yq, zq), ORC_INF);
                    for (int64_t l = 0; l < nk; ++l)
                        if (kcap[l] > 0 && z - l >= 0) add_arc(g, mode, v, idx3(Y, Z, xq, yq, z - l), kcap[l]);
                }
            }
}

static void graph_free(orc_graph *g) {
    free(g->first);
    free(g->head);
    free(g->rev);
    free(g->cap);
    free(g->cap0);
    free(g->fill);
    memset(g, 0, sizeof *g);
}

static int graph_build(orc_graph *g, const int32_t *c, int32_t X, int32_t Y, int32_t Z,
                       int32_t delta, const int64_t *kcap, int32_t nk, int keep_cap0) {
    memset(g, 0, sizeof *g);
    const int64_t N = (int64_t)X * Y * Z;
    g->n = N + 2;
    g->first = calloc((size_t)g->n + 1, sizeof(int64_t));
    if (!g->first) return ORC_E_NOMEM;
    enumerate_arcs(g, 0, c, X, Y, Z, delta, kcap, nk);
    for (int64_t i = 0; i < g->n; ++i) g->first[i + 1] += g->first[i];
    g->m = g->first[g->n];
    g->head = malloc((size_t)g->m * sizeof(int32_t));
    g->rev = malloc((size_t)g->m * sizeof(int64_t));
    g->cap = malloc((size_t)g->m * sizeof(int64_t));
    g->fill = malloc((size_t)g->n * sizeof(int64_t));
    if (keep_cap0) g->cap0 = malloc((size_t)g->m * sizeof(int64_t));
    if (!g->head || !g->rev || !g->cap || !g->fill || (keep_cap0 && !g->cap0)) {
        graph_free(g);
        return ORC_E_NOMEM;
    }
    memcpy(g->fill, g->first, (size_t)g->n * sizeof(int64_t));
    enumerate_arcs(g, 1, c, X, Y, Z, delta, kcap, nk);
    free(g->fill);
    g->fill = NULL;
    return ORC_OK;
}

/* Dinic (Section 2): BFS levels from s over residual arcs, then a blocking flow of
 * shortest augmenting paths found by depth-first search with a current-arc pointer
 * per node; repeat until t is unreachable. */
typedef struct {
    int32_t *level;
    int64_t *queue;
    int64_t *iter;
    int64_t *path;
    int64_t phases;
    int64_t augmentations;
} orc_dinic;

static int dinic_bfs(const orc_graph *g, orc_dinic *d, int64_t s, int64_t t) {
    for (int64_t i = 0; i < g->n; ++i) d->level[i] = -1;
    int64_t qh = 0, qt = 0;
    d->level[s] = 0;
    d->queue[qt++] = s;
    while (qh < qt) {
        const int64_t u = d->queue[qh++];
        for (int64_t a = g->first[u]; a < g->first[u + 1]; ++a) {
            const int64_t v = g->head[a];
            if (g->cap[a] > 0 && d->level[v] < 0) {
                d->level[v] = d->level[u] + 1;
                d->queue[qt++] = v;
            }
        }
        /* Every node closer to s than t is labelled once t is; nodes left unlabelled
         * lie at t's distance or beyond and can be on no shortest s-t path. */
        if (d->level[t] >= 0) break;
    }
    return d->level[t] >= 0;
}

static int64_t dinic_blocking_flow(orc_graph *g, orc_dinic *d, int64_t s, int64_t t) {
    int64_t total = 0, depth = 0, u = s;
    memcpy(d->iter, g->first, (size_t)g->n * sizeof(int64_t));
    for (;;) {
        if (u == t) {
            int64_t b = ORC_INF;
            for (int64_t k = 0; k < depth; ++k)
                if (g->cap[d->path[k]] < b) b = g->cap[d->path[k]];
            int64_t cut_at = -1;
            for (int64_t k = 0; k < depth; ++k) {
                const int64_t a = d->path[k];
                g->cap[a] -= b;
                g->cap[g->rev[a]] += b;
                if (cut_at < 0 && g->cap[a] == 0) cut_at = k;
            }
            total += b;
            d->augmentations++;
            /* resume from the tail of the first arc this augmentation saturated */
            depth = cut_at;
            u = (depth == 0) ? s : g->head[d->path[depth - 1]];
            continue;
        }
        int64_t a = d->iter[u];
        for (; a < g->first[u + 1]; ++a) {
            const int64_t v = g->head[a];
            if (g->cap[a] > 0 && d->level[v] == d->level[u] + 1) break;
        }
        d->iter[u] = a;
        if (a < g->first[u + 1]) {
            d->path[depth++] = a;
            u = g->head[a];
        } else {
            d->level[u] = -1; /* dead end for this phase */
            if (u == s) break;
            const int64_t back = d->path[--depth];
            u = g->head[g->rev[back]];
            d->iter[u]++;
        }
    }
    return total;
}

/* Nodes reachable from s over residual arcs: the source side of the minimal min cut. */
static void residual_reach(const orc_graph *g, int64_t s, uint8_t *in_s, int64_t *queue) {
    memset(in_s, 0, (size_t)g->n);
    int64_t qh = 0, qt = 0;
    in_s[s] = 1;
    queue[qt++] = s;
    while (qh < qt) {
        const int64_t u = queue[qh++];
        for (int64_t a = g->first[u]; a < g->first[u + 1]; ++a) {
            const int64_t v = g->head[a];
            if (g->cap[a] > 0 && !in_s[v]) {
                in_s[v] = 1;
                queue[qt++] = v;
            }
        }
    }
}

/* Capacity (Eq. 2), antisymmetric bookkeeping (Eq. 3) and conservation (Eq. 4) of the
 * final flow, and max-flow = min-cut (Theorem 1.1) on the cut found. */
static int check_invariants(const orc_graph *g, int64_t s, int64_t t, const uint8_t *in_s,
                            int64_t flow) {
    int64_t *net = calloc((size_t)g->n, sizeof(int64_t));
    if (!net) return ORC_E_NOMEM;
    int64_t cut = 0;
    int rc = ORC_OK;
    for (int64_t u = 0; u < g->n && rc == ORC_OK; ++u)
        for (int64_t a = g->first[u]; a < g->first[u + 1]; ++a) {
            const int64_t f = g->cap0[a] - g->cap[a]; /* flow on this half-arc */
            if (g->cap[a] < 0 || f > g->cap0[a]) { rc = ORC_E_CAPACITY; break; }
            if (f != -(g->cap0[g->rev[a]] - g->cap[g->rev[a]])) { rc = ORC_E_CAPACITY; break; }
            net[u] -= f; /* f > 0 leaves u; f < 0 on a reverse half-arc enters u */
            if (in_s[u] && !in_s[g->head[a]]) cut += g->cap0[a];
        }
    if (rc == ORC_OK) {
        for (int64_t v = 0; v < g->n; ++v)
            if (v != s && v != t && net[v] != 0) { rc = ORC_E_CONSERVATION; break; }
        if (rc == ORC_OK && (net[t] != flow || net[s] != -flow)) rc = ORC_E_CONSERVATION;
        if (rc == ORC_OK && cut != flow) rc = ORC_E_CUT;
    }
    free(net);
    return rc;
}

/*
 * Solve one volume. cost: int32 [X][Y][Z] (z fastest). heights_out: int32 [X*Y],
 * column (x,y) at x*Y + y. stats_out (may be NULL): phases, augmentations, nodes,
 * half-arcs. check != 0 keeps the initial capacities and verifies Eq. 2-4 and
 * Theorem 1.1 on the result.
 */
static int solve_layers(const int32_t *cost, int32_t X, int32_t Y, int32_t Z, int32_t delta,
                        const int64_t *kcap, int32_t nk, int32_t check, int64_t *flow_out,
                        int32_t *heights_out, int64_t *stats_out) {
    if ((int64_t)X * Y * Z + 2 > INT32_MAX) return ORC_E_ARGS;
    orc_graph g;
    int rc = graph_build(&g, cost, X, Y, Z, delta, kcap, nk, check != 0);
    if (rc != ORC_OK) return rc;
    const int64_t N = (int64_t)X * Y * Z, s = N, t = N + 1;
    orc_dinic d = {0};
    d.level = malloc((size_t)g.n * sizeof(int32_t));
    d.queue = malloc((size_t)g.n * sizeof(int64_t));
    d.iter = malloc((size_t)g.n * sizeof(int64_t));
    d.path = malloc((size_t)g.n * sizeof(int64_t));
    uint8_t *in_s = malloc((size_t)g.n);
    if (!d.level || !d.queue || !d.iter || !d.path || !in_s) {
        rc = ORC_E_NOMEM;
        goto done;
    }
    int64_t flow = 0;
    while (dinic_bfs(&g, &d, s, t)) {
        d.phases++;
        flow += dinic_blocking_flow(&g, &d, s, t);
    }
    residual_reach(&g, s, in_s, d.queue);
    for (int64_t col = 0; col < (int64_t)X * Y; ++col) {
        int32_t h = -1;
        for (int64_t z = 0; z < Z; ++z)
            if (in_s[col * Z + z]) h = (int32_t)z;
        heights_out[col] = h;
        if (h < 0) rc = ORC_E_SURFACE;
    }
    if (rc == ORC_OK && check) rc = check_invariants(&g, s, t, in_s, flow);
    *flow_out = flow;
    if (stats_out) {
        stats_out[0] = d.phases;
        stats_out[1] = d.augmentations;
        stats_out[2] = g.n;
        stats_out[3] = g.m;
    }
done:
    free(d.level);
    free(d.queue);
    free(d.iter);
    free(d.path);
    free(in_s);
    graph_free(&g);
    return rc;
}

int oracle_solve(const int32_t *cost, int32_t X, int32_t Y, int32_t Z, int32_t delta,
                 int64_t alpha, int32_t check, int64_t *flow_out, int32_t *heights_out,
                 int64_t *stats_out) {
    if (!cost || X < 1 || Y < 1 || Z < 1 || delta < 0 || alpha < 0 || !flow_out || !heights_out)
        return ORC_E_ARGS;
    return solve_layers(cost, X, Y, Z, delta, &alpha, 1, check, flow_out, heights_out, stats_out);
}

/* Layer capacities k_0 = f(1), k_d = f(d+1) - 2 f(d) + f(d-1) of a convex pairwise cost
 * given as f[0..delta-1] = f(1..delta) (f(0) = 0). Returns 0 when f is not convex or
 * f(1) < 0. */
static int convex_layers(const int64_t *f, int32_t delta, int64_t *kcap) {
    for (int32_t d = 0; d < delta; ++d) {
        const int64_t fd = d == 0 ? 0 : f[d - 1];
        const int64_t fm = d <= 1 ? 0 : f[d - 2];
        kcap[d] = d == 0 ? f[0] : f[d] - 2 * fd + fm;
        if (kcap[d] < 0) return 0;
    }
    return 1;
}

/*
 * Solve one volume with the convex pairwise cost f (f[0..delta-1] = f(1..delta), f(0) = 0):
 * minimise sum_col c(col, h(col)) + sum over unordered 4-neighbour pairs f(|h_p - h_q|)
 * subject to |h_p - h_q| <= delta. Outputs as oracle_solve. ORC_E_ARGS when f is not
 * convex (a negative second difference, or f(1) < 0).
 */
int oracle_solve_convex(const int32_t *cost, int32_t X, int32_t Y, int32_t Z, int32_t delta,
                        const int64_t *f, int32_t check, int64_t *flow_out, int32_t *heights_out,
                        int64_t *stats_out) {
    if (!cost || X < 1 || Y < 1 || Z < 1 || delta < 0 || (delta > 0 && !f) || !flow_out || !heights_out)
        return ORC_E_ARGS;
    int64_t *kcap = malloc(((size_t)delta + 1) * sizeof(int64_t));
    if (!kcap) return ORC_E_NOMEM;
    int rc = convex_layers(f, delta, kcap)
                 ? solve_layers(cost, X, Y, Z, delta, kcap, delta, check, flow_out, heights_out, stats_out)
                 : ORC_E_ARGS;
    free(kcap);
    return rc;
}

/*
 * Surface energy with the convex pairwise cost, from its definition:
 * E = sum_col c(col, h(col)) + sum over unordered 4-neighbour pairs f(|h_p - h_q|).
 * *feasible is set to 0 if some pair differs by more than delta or a height is outside
 * [0, Z) (those pairs add nothing).
 */
int64_t oracle_energy_convex(const int32_t *cost, int32_t X, int32_t Y, int32_t Z, int32_t delta,
                             const int64_t *f, const int32_t *h, int32_t *feasible) {
    int64_t e = 0;
    int ok = 1;
    for (int64_t x = 0; x < X; ++x)
        for (int64_t y = 0; y < Y; ++y) {
            const int64_t hp = h[x * Y + y];
            if (hp < 0 || hp >= Z) { ok = 0; continue; }
            e += cost[idx3(Y, Z, x, y, hp)];
            for (int k = 0; k < 2; ++k) {
                const int64_t xq = x + (k == 0), yq = y + (k == 1);
                if (xq >= X || yq >= Y) continue;
                const int64_t dq = hp - h[xq * Y + yq];
                const int64_t ad = dq < 0 ? -dq : dq;
                if (ad > delta) { ok = 0; continue; }
                if (ad > 0) e += f[ad - 1];
            }
        }
    if (feasible) *feasible = ok;
    return e;
}

/*
 * Solve one volume as oracle_solve does and describe the final flow in the layout of a
 * solver state (the arrays oracle_certify takes, include/pog.h's export), so that the
 * certificate can be checked on a state known to be optimal. The literal graph keeps the
 * bottom layer z = 0 as nodes; the exported state treats it as part of the source, so
 * for every node v above it:
 *   sink   = residual capacity of v -> t,
 *   excess = unused capacity of s -> v (the state has every source arc saturated) plus
 *            the flow v sends into bottom-layer nodes (arcs that the state does not keep),
 *   fdown  = flow on v -> (x,y,z-1) for z >= 2, fhard[d] = flow on the hard arc towards
 *            neighbour d when it lands at z - delta >= 1, gsoft[k] = flow v -> q minus
 *            flow q -> v for the neighbour q at x+1 (k = 0) or y+1 (k = 1),
 *   in_cut = 1 for the nodes reachable from s in the final residual graph.
 * Arcs are told apart by their heads and initial capacities (infinite or alpha).
 */
int oracle_solve_state(const int32_t *cost, int32_t X, int32_t Y, int32_t Z, int32_t delta, int64_t alpha,
                       int64_t *flow_out, int32_t *heights_out, int32_t *excess, int32_t *sink, int32_t *fdown,
                       int32_t *fhard, int32_t *gsoft, int32_t *in_cut) {
    if (!cost || X < 1 || Y < 1 || Z < 1 || delta < 0 || alpha < 0 || !flow_out || !heights_out || !excess ||
        !sink || !fdown || !fhard || !gsoft || !in_cut)
        return ORC_E_ARGS;
    if ((int64_t)X * Y * Z + 2 > INT32_MAX) return ORC_E_ARGS;
    orc_graph g;
    int rc = graph_build(&g, cost, X, Y, Z, delta, &alpha, 1, 1);
    if (rc != ORC_OK) return rc;
    const int64_t N = (int64_t)X * Y * Z, s = N, t = N + 1;
    orc_dinic d = {0};
    d.level = malloc((size_t)g.n * sizeof(int32_t));
    d.queue = malloc((size_t)g.n * sizeof(int64_t));
    d.iter = malloc((size_t)g.n * sizeof(int64_t));
    d.path = malloc((size_t)g.n * sizeof(int64_t));
    uint8_t *in_s = malloc((size_t)g.n);
    int64_t *acc = calloc((size_t)N * 9, sizeof(int64_t)); /* excess, fdown, fhard[4], gsoft[2], sink */
    if (!d.level || !d.queue || !d.iter || !d.path || !in_s || !acc) {
        rc = ORC_E_NOMEM;
        goto done;
    }
    int64_t flow = 0;
    while (dinic_bfs(&g, &d, s, t)) flow += dinic_blocking_flow(&g, &d, s, t);
    residual_reach(&g, s, in_s, d.queue);
    int64_t *exc = acc, *fdn = acc + N, *fh = acc + 2 * N, *gs = acc + 6 * N, *snk = acc + 8 * N;
    /* source arcs: the unused capacity stays at the node as excess */
    for (int64_t a = g.first[s]; a < g.first[s + 1]; ++a) {
        const int64_t v = g.head[a];
        if (g.cap0[a] > 0 && v % Z != 0) exc[v] += g.cap[a];
    }
    for (int64_t u = 0; u < N; ++u) {
        const int64_t z = u % Z, col = u / Z, x = col / Y, y = col % Y;
        if (z == 0) continue;
        for (int64_t a = g.first[u]; a < g.first[u + 1]; ++a) {
            if (g.cap0[a] <= 0) continue; /* a reverse half-arc */
            const int64_t h = g.head[a], f = g.cap0[a] - g.cap[a];
            if (h == t) {
                snk[u] = g.cap[a];
                continue;
            }
            const int64_t hz = h % Z, hcol = h / Z, hx = hcol / Y, hy = hcol % Y;
            if (hz == 0) { /* into the bottom layer: not an arc of the state */
                exc[u] += f;
                continue;
            }
            if (hcol == col) { /* the column arc (x,y,z) -> (x,y,z-1) */
                fdn[u] += f;
                continue;
            }
            int dir = -1;
            for (int k = 0; k < 4; ++k)
                if (hx == x + DX[k] && hy == y + DY[k]) dir = k;
            if (dir < 0) {
                rc = ORC_E_ARGS;
                goto done;
            }
            if (g.cap0[a] == ORC_INF) { /* hard arc landing at z - delta >= 1 */
                fh[dir * N + u] += f;
            } else if (dir & 1) { /* soft arc towards x+1 / y+1 */
                gs[(dir >> 1) * N + u] += f;
            } else { /* soft arc towards x-1 / y-1: counts against the neighbour's pair */
                gs[(dir >> 1) * N + h] -= f;
            }
        }
    }
    for (int64_t v = 0; v < N; ++v) {
        const int bottom = v % Z == 0;
        excess[v] = bottom ? 0 : (int32_t)exc[v];
        sink[v] = bottom ? 0 : (int32_t)snk[v];
        fdown[v] = bottom ? 0 : (int32_t)fdn[v];
        for (int k = 0; k < 4; ++k) fhard[k * N + v] = bottom ? 0 : (int32_t)fh[k * N + v];
        for (int k = 0; k < 2; ++k) gsoft[k * N + v] = bottom ? 0 : (int32_t)gs[k * N + v];
        in_cut[v] = in_s[v];
    }
    for (int64_t col = 0; col < (int64_t)X * Y; ++col) {
        int32_t hgt = -1;
        for (int64_t z = 0; z < Z; ++z)
            if (in_s[col * Z + z]) hgt = (int32_t)z;
        heights_out[col] = hgt;
        if (hgt < 0) rc = ORC_E_SURFACE;
    }
    *flow_out = flow;
done:
    free(d.level);
    free(d.queue);
    free(d.iter);
    free(d.path);
    free(in_s);
    free(acc);
    graph_free(&g);
    return rc;
}

/*
 * Surface energy of Eq. 1 for a height map: E = sum_col c(col, h(col)) +
 * alpha * sum over unordered 4-neighbour pairs |h_p - h_q|. *feasible is set to 0 if
 * some pair differs by more than delta or a height is outside [0, Z).
 */
int64_t oracle_energy(const int32_t *cost, int32_t X, int32_t Y, int32_t Z, int32_t delta,
                      int64_t alpha, const int32_t *h, int32_t *feasible) {
    int64_t e = 0;
    int ok = 1;
    for (int64_t x = 0; x < X; ++x)
        for (int64_t y = 0; y < Y; ++y) {
            const int64_t hp = h[x * Y + y];
            if (hp < 0 || hp >= Z) { ok = 0; continue; }
            e += cost[idx3(Y, Z, x, y, hp)];
            if (x + 1 < X) {
                const int64_t dq = hp - h[(x + 1) * Y + y];
                const int64_t ad = dq < 0 ? -dq : dq;
                if (ad > delta) ok = 0;
                e += alpha * ad;
            }
            if (y + 1 < Y) {
                const int64_t dq = hp - h[x * Y + y + 1];
                const int64_t ad = dq < 0 ? -dq : dq;
                if (ad > delta) ok = 0;
                e += alpha * ad;
            }
        }
    if (feasible) *feasible = ok;
    return e;
}

/*
 * Capacity (Eq. 6) of the s-t cut whose source side is {s} and, in each column, the
 * nodes z <= h(col), counted arc by arc over the literal graph. Returns -1 when an
 * infinite arc crosses the cut (the surface violates the hard constraints).
 */
int64_t oracle_cut_capacity(const int32_t *cost, int32_t X, int32_t Y, int32_t Z,
                            int32_t delta, int64_t alpha, const int32_t *h) {
    const int64_t bsum = bottom_layer_sum(cost, X, Y, Z);
    int64_t cut = 0;
    for (int64_t x = 0; x < X; ++x)
        for (int64_t y = 0; y < Y; ++y)
            for (int64_t z = 0; z < Z; ++z) {
                const int in_u = z <= h[x * Y + y];
                const int64_t w = node_weight(cost, X, Y, Z, x, y, z, bsum);
                if (w < 0 && !in_u) cut += -w;          /* s -> v with v outside */
                if (w > 0 && in_u) cut += w;            /* v -> t with v inside  */
                if (!in_u) continue;
                if (z >= 1 && !(z - 1 <= h[x * Y + y])) return -1;
                for (int d = 0; d < 4; ++d) {
                    const int64_t xq = x + DX[d], yq = y + DY[d];
                    if (xq < 0 || xq >= X || yq < 0 || yq >= Y) continue;
                    const int64_t zq = (z - delta > 0) ? z - delta : 0;
                    if (!(zq <= h[xq * Y + yq])) return -1;
                    if (alpha > 0 && !(z <= h[xq * Y + yq])) cut += alpha;
                }
            }
    return cut;
}

/*
 * Optimality certificate of a solver's final residual state, for volumes too large for
 * Dinic. The state is the one include/pog.h exports (int32 arrays of N = X*Y*Z nodes,
 * z fastest): excess, sink residual, flow on the down arc, flow on the hard arc of each
 * direction d (fhard[d*N + v]), net soft flow towards x+1 / y+1 (gsoft[k*N + v]), the
 * cut marks, and the heights. In that state the bottom layer z = 0 is merged into the
 * source: it is in every minimum cut (its weights sum to -1 and every non-empty closed
 * set contains it), so arcs into it carry no flow and its sink arcs add
 * sum_{z=0, w>0} w to the flow value.
 *
 * Checks, in order (return code):
 *   capacity (Eq. 2) of every arc and sink arc, zero flow on absent arcs      -> 10
 *   excess = inflow - outflow (Eq. 4 relaxed to a preflow) and excess >= 0     -> 11
 *   flow value (Eq. 5) of the preflow equals `flow`                          -> 12
 *   the cut marks equal the residual reach of the nodes with excess           -> 13
 *   each height is the top marked node of its column (0 if none)              -> 14
 *   the capacity (Eq. 6) of the cut below the heights equals `flow`           -> 15
 * The last check with a feasible preflow of value `flow` proves both optimal
 * (Theorem 1.1); the reach check proves the cut is the minimal one.
 */
int oracle_certify(const int32_t *cost, int32_t X, int32_t Y, int32_t Z, int32_t delta, int64_t alpha,
                   const int32_t *excess, const int32_t *sink, const int32_t *fdown, const int32_t *fhard,
                   const int32_t *gsoft, const int32_t *in_cut, const int32_t *heights, int64_t flow) {
    const int64_t N = (int64_t)X * Y * Z;
    const int64_t bsum = bottom_layer_sum(cost, X, Y, Z);
    int64_t *net = calloc((size_t)N, sizeof(int64_t));
    uint8_t *seen = calloc((size_t)N, 1);
    int64_t *queue = malloc((size_t)N * sizeof(int64_t));
    int rc = ORC_OK;
    if (!net || !seen || !queue) {
        rc = ORC_E_NOMEM;
        goto out;
    }
    int64_t value = 0;
    for (int64_t x = 0; x < X; ++x)
        for (int64_t y = 0; y < Y; ++y)
            for (int64_t z = 0; z < Z; ++z) {
                const int64_t v = idx3(Y, Z, x, y, z);
                const int64_t w = node_weight(cost, X, Y, Z, x, y, z, bsum);
                if (z == 0) { /* part of the source: no state of its own */
                    if (w > 0) value += w;
                    if (sink[v] != 0 || fdown[v] != 0 || excess[v] != 0) { rc = 10; goto out; }
                    for (int d = 0; d < 4; ++d)
                        if (fhard[d * N + v] != 0 || (alpha > 0 && gsoft && d < 2 && gsoft[d * N + v] != 0)) {
                            rc = 10;
                            goto out;
                        }
                    continue;
                }
                const int64_t snk0 = w > 0 ? w : 0;
                if (sink[v] < 0 || sink[v] > snk0) { rc = 10; goto out; }
                net[v] += (w < 0 ? -w : 0) - (snk0 - sink[v]);
                value += snk0 - sink[v];
                if (z >= 2) {
                    if (fdown[v] < 0) { rc = 10; goto out; }
                    net[v] -= fdown[v];
                    net[v - 1] += fdown[v];
                } else if (fdown[v] != 0) { rc = 10; goto out; }
                for (int d = 0; d < 4; ++d) {
                    const int64_t xq = x + DX[d], yq = y + DY[d];
                    const int64_t f = fhard[d * N + v];
                    const int in_grid = xq >= 0 && xq < X && yq >= 0 && yq < Y;
                    if (in_grid && z - delta >= 1) {
                        if (f < 0) { rc = 10; goto out; }
                        const int64_t head = idx3(Y, Z, xq, yq, z - delta);
                        net[v] -= f;
                        net[head] += f;
                    } else if (f != 0) { rc = 10; goto out; }
                    if (alpha > 0 && gsoft && (d & 1)) { /* the pair towards x+1 / y+1 */
                        const int64_t g = gsoft[(d >> 1) * N + v];
                        if (in_grid) {
                            if (g < -alpha || g > alpha) { rc = 10; goto out; }
                            net[v] -= g;
                            net[idx3(Y, Z, xq, yq, z)] += g;
                        } else if (g != 0) { rc = 10; goto out; }
                    }
                }
            }
    for (int64_t v = 0; v < N; ++v) {
        if (v % Z == 0) continue;
        if (net[v] != excess[v] || excess[v] < 0) { rc = 11; goto out; }
    }
    if (value != flow) { rc = 12; goto out; }
    /* residual reach of the excess nodes (z >= 1 only; the bottom layer is the source) */
    int64_t qh = 0, qt = 0;
    for (int64_t v = 0; v < N; ++v)
        if (v % Z != 0 && excess[v] > 0) { seen[v] = 1; queue[qt++] = v; }
    while (qh < qt) {
        const int64_t u = queue[qh++];
        const int64_t z = u % Z, col = u / Z, x = col / Y, y = col % Y;
        int64_t nbr[16];
        int k = 0;
        if (z >= 2) nbr[k++] = u - 1;                      /* down arc: infinite */
        if (z + 1 < Z && fdown[u + 1] > 0) nbr[k++] = u + 1; /* reverse of the up node's down arc */
        for (int d = 0; d < 4; ++d) {
            const int64_t xq = x + DX[d], yq = y + DY[d];
            if (xq < 0 || xq >= X || yq < 0 || yq >= Y) continue;
            if (z - delta >= 1) nbr[k++] = idx3(Y, Z, xq, yq, z - delta); /* hard arc: infinite */
            if (z + delta < Z) {                                        /* reverse of a hard arc into u */
                const int64_t w = idx3(Y, Z, xq, yq, z + delta);
                if (fhard[(d ^ 1) * N + w] > 0) nbr[k++] = w;
            }
            if (alpha > 0 && gsoft) {
                const int64_t q = idx3(Y, Z, xq, yq, z);
                const int64_t g = (d & 1) ? gsoft[(d >> 1) * N + u] : -gsoft[(d >> 1) * N + q];
                if (alpha - g > 0) nbr[k++] = q; /* g: net flow u -> q */
            }
        }
        for (int i = 0; i < k; ++i)
            if (!seen[nbr[i]]) { seen[nbr[i]] = 1; queue[qt++] = nbr[i]; }
    }
    for (int64_t v = 0; v < N; ++v) {
        if (v % Z == 0) continue;
        if ((in_cut[v] != 0) != (seen[v] != 0)) { rc = 13; goto out; }
    }
    for (int64_t col = 0; col < (int64_t)X * Y; ++col) {
        int32_t top = 0;
        for (int64_t z = 1; z < Z; ++z)
            if (in_cut[col * Z + z]) top = (int32_t)z;
        if (heights[col] != top) { rc = 14; goto out; }
    }
    if (oracle_cut_capacity(cost, X, Y, Z, delta, alpha, heights) != flow) rc = 15;
out:
    free(net);
    free(seen);
    free(queue);
    return rc;
}

/* ------------------------------------------------------------------------------------------
 * Convex pairwise costs: the oracle's own final flow in a solver-state layout, the literal
 * cut capacity of a surface, and the O(N) certificate of a state.
 *
 * State layout (int32 arrays, z fastest, N = X*Y*Z, the bottom layer merged into the source as
 * in oracle_solve_state): excess, sink, fdown, fhard[4N] as there; gpair[2N] = net flow of the
 * d = 0 layer from v to its neighbour at x+1 (k = 0) or y+1 (k = 1), in [-k_0, k_0];
 * flayer[((d-1)*4 + dir)*N + v] = flow on the layer-d arc from v to its neighbour in direction
 * dir at height z - d (present when z - d >= 1 and k_d > 0), d = 1 .. delta-1; in_cut.
 * ------------------------------------------------------------------------------------------ */

/* Capacity (Eq. 6) of the cut whose source side is {s} and, in each column, the nodes
 * z <= h(col), counted arc by arc over the literal layered graph; -1 when an infinite arc
 * crosses it. f as for oracle_solve_convex. */
int64_t oracle_cut_capacity_convex(const int32_t *cost, int32_t X, int32_t Y, int32_t Z, int32_t delta,
                                   const int64_t *f, const int32_t *h) {
    int64_t *kcap = malloc(((size_t)delta + 1) * sizeof(int64_t));
    if (!kcap) return -2;
    if (!convex_layers(f, delta, kcap)) {
        free(kcap);
        return -2;
    }
    const int64_t bsum = bottom_layer_sum(cost, X, Y, Z);
    int64_t cut = 0;
    for (int64_t x = 0; x < X; ++x)
        for (int64_t y = 0; y < Y; ++y)
            for (int64_t z = 0; z < Z; ++z) {
                const int in_u = z <= h[x * Y + y];
                const int64_t w = node_weight(cost, X, Y, Z, x, y, z, bsum);
                if (w < 0 && !in_u) cut += -w;
                if (w > 0 && in_u) cut += w;
                if (!in_u) continue;
                if (z >= 1 && !(z - 1 <= h[x * Y + y])) { cut = -1; goto done; }
                for (int d = 0; d < 4; ++d) {
                    const int64_t xq = x + DX[d], yq = y + DY[d];
                    if (xq < 0 || xq >= X || yq < 0 || yq >= Y) continue;
                    const int64_t hq = h[xq * Y + yq];
                    const int64_t zq = (z - delta > 0) ? z - delta : 0;
                    if (!(zq <= hq)) { cut = -1; goto done; }
                    for (int64_t l = 0; l < delta; ++l)
                        if (kcap[l] > 0 && z - l >= 0 && !(z - l <= hq)) cut += kcap[l];
                }
            }
done:
    free(kcap);
    return cut;
}

int oracle_solve_state_convex(const int32_t *cost, int32_t X, int32_t Y, int32_t Z, int32_t delta, const int64_t *f,
                              int64_t *flow_out, int32_t *heights_out, int32_t *excess, int32_t *sink,
                              int32_t *fdown, int32_t *fhard, int32_t *gpair, int32_t *flayer, int32_t *in_cut) {
    if (!cost || X < 1 || Y < 1 || Z < 1 || delta < 0 || (delta > 0 && !f) || !flow_out || !heights_out ||
        !excess || !sink || !fdown || !fhard || !gpair || (delta > 1 && !flayer) || !in_cut)
        return ORC_E_ARGS;
    if ((int64_t)X * Y * Z + 2 > INT32_MAX) return ORC_E_ARGS;
    int64_t *kcap = malloc(((size_t)delta + 1) * sizeof(int64_t));
    if (!kcap) return ORC_E_NOMEM;
    if (!convex_layers(f, delta, kcap)) {
        free(kcap);
        return ORC_E_ARGS;
    }
    orc_graph g;
    int rc = graph_build(&g, cost, X, Y, Z, delta, kcap, delta, 1);
    if (rc != ORC_OK) {
        free(kcap);
        return rc;
    }
    const int64_t N = (int64_t)X * Y * Z, s = N, t = N + 1;
    const int64_t nl = delta > 1 ? delta - 1 : 0;
    orc_dinic d = {0};
    d.level = malloc((size_t)g.n * sizeof(int32_t));
    d.queue = malloc((size_t)g.n * sizeof(int64_t));
    d.iter = malloc((size_t)g.n * sizeof(int64_t));
    d.path = malloc((size_t)g.n * sizeof(int64_t));
    uint8_t *in_s = malloc((size_t)g.n);
    int64_t *acc = calloc((size_t)N * (9 + 4 * nl), sizeof(int64_t)); /* excess fdown fhard[4] gpair[2] sink flayer */
    if (!d.level || !d.queue || !d.iter || !d.path || !in_s || !acc) {
        rc = ORC_E_NOMEM;
        goto done;
    }
    int64_t flow = 0;
    while (dinic_bfs(&g, &d, s, t)) flow += dinic_blocking_flow(&g, &d, s, t);
    residual_reach(&g, s, in_s, d.queue);
    int64_t *exc = acc, *fdn = acc + N, *fh = acc + 2 * N, *gp = acc + 6 * N, *snk = acc + 8 * N, *fl = acc + 9 * N;
    for (int64_t a = g.first[s]; a < g.first[s + 1]; ++a) {
        const int64_t v = g.head[a];
        if (g.cap0[a] > 0 && v % Z != 0) exc[v] += g.cap[a];
    }
    for (int64_t u = 0; u < N; ++u) {
        const int64_t z = u % Z, col = u / Z, x = col / Y, y = col % Y;
        if (z == 0) continue;
        for (int64_t a = g.first[u]; a < g.first[u + 1]; ++a) {
            if (g.cap0[a] <= 0) continue; /* a reverse half-arc */
            const int64_t h = g.head[a], fa = g.cap0[a] - g.cap[a];
            if (h == t) {
                snk[u] = g.cap[a];
                continue;
            }
            const int64_t hz = h % Z, hcol = h / Z, hx = hcol / Y, hy = hcol % Y;
            if (hz == 0) { /* into the bottom layer: not an arc of the state */
                exc[u] += fa;
                continue;
            }
            if (hcol == col) {
                fdn[u] += fa;
                continue;
            }
            int dir = -1;
            for (int k = 0; k < 4; ++k)
                if (hx == x + DX[k] && hy == y + DY[k]) dir = k;
            if (dir < 0) {
                rc = ORC_E_ARGS;
                goto done;
            }
            const int64_t drop = z - hz;
            if (g.cap0[a] == ORC_INF) {
                fh[dir * N + u] += fa;
            } else if (drop == 0) {
                if (dir & 1) gp[(dir >> 1) * N + u] += fa;
                else gp[(dir >> 1) * N + h] -= fa;
            } else if (drop >= 1 && drop < delta) {
                fl[((drop - 1) * 4 + dir) * N + u] += fa;
            } else {
                rc = ORC_E_ARGS;
                goto done;
            }
        }
    }
    for (int64_t v = 0; v < N; ++v) {
        const int bottom = v % Z == 0;
        excess[v] = bottom ? 0 : (int32_t)exc[v];
        sink[v] = bottom ? 0 : (int32_t)snk[v];
        fdown[v] = bottom ? 0 : (int32_t)fdn[v];
        for (int k = 0; k < 4; ++k) fhard[k * N + v] = bottom ? 0 : (int32_t)fh[k * N + v];
        for (int k = 0; k < 2; ++k) gpair[k * N + v] = bottom ? 0 : (int32_t)gp[k * N + v];
        for (int64_t j = 0; j < 4 * nl; ++j) flayer[j * N + v] = bottom ? 0 : (int32_t)fl[j * N + v];
        in_cut[v] = in_s[v];
    }
    for (int64_t col = 0; col < (int64_t)X * Y; ++col) {
        int32_t hgt = -1;
        for (int64_t z = 0; z < Z; ++z)
            if (in_s[col * Z + z]) hgt = (int32_t)z;
        heights_out[col] = hgt;
        if (hgt < 0) rc = ORC_E_SURFACE;
    }
    *flow_out = flow;
done:
    free(d.level);
    free(d.queue);
    free(d.iter);
    free(d.path);
    free(in_s);
    free(acc);
    free(kcap);
    graph_free(&g);
    return rc;
}

/*
 * Optimality certificate of a convex-cost state (layout above), the checks and return codes
 * of oracle_certify: capacity of every arc and sink arc with zero flow on absent arcs (10),
 * excess = inflow - outflow >= 0 (11), the preflow's value equals `flow` (12), the cut marks
 * equal the residual reach of the nodes with excess (13), each height is the top marked node
 * of its column (14), and the literal capacity of the cut below the heights equals `flow`
 * (15). ORC_E_ARGS when f is not convex.
 */
int oracle_certify_convex(const int32_t *cost, int32_t X, int32_t Y, int32_t Z, int32_t delta, const int64_t *f,
                          const int32_t *excess, const int32_t *sink, const int32_t *fdown, const int32_t *fhard,
                          const int32_t *gpair, const int32_t *flayer, const int32_t *in_cut, const int32_t *heights,
                          int64_t flow) {
    const int64_t N = (int64_t)X * Y * Z;
    const int64_t nl = delta > 1 ? delta - 1 : 0;
    const int64_t bsum = bottom_layer_sum(cost, X, Y, Z);
    int64_t *kcap = malloc(((size_t)delta + 1) * sizeof(int64_t));
    int64_t *net = calloc((size_t)N, sizeof(int64_t));
    uint8_t *seen = calloc((size_t)N, 1);
    int64_t *queue = malloc((size_t)N * sizeof(int64_t));
    int rc = ORC_OK;
    if (!kcap || !net || !seen || !queue) {
        rc = ORC_E_NOMEM;
        goto out;
    }
    if (!convex_layers(f, delta, kcap)) {
        rc = ORC_E_ARGS;
        goto out;
    }
    const int64_t k0 = delta > 0 ? kcap[0] : 0;
    int64_t value = 0;
    for (int64_t x = 0; x < X; ++x)
        for (int64_t y = 0; y < Y; ++y)
            for (int64_t z = 0; z < Z; ++z) {
                const int64_t v = idx3(Y, Z, x, y, z);
                const int64_t w = node_weight(cost, X, Y, Z, x, y, z, bsum);
                if (z == 0) { /* part of the source: no state of its own */
                    if (w > 0) value += w;
                    if (sink[v] != 0 || fdown[v] != 0 || excess[v] != 0) { rc = 10; goto out; }
                    for (int d = 0; d < 4; ++d)
                        if (fhard[d * N + v] != 0 || (d < 2 && gpair[d * N + v] != 0)) { rc = 10; goto out; }
                    for (int64_t j = 0; j < 4 * nl; ++j)
                        if (flayer[j * N + v] != 0) { rc = 10; goto out; }
                    continue;
                }
                const int64_t snk0 = w > 0 ? w : 0;
                if (sink[v] < 0 || sink[v] > snk0) { rc = 10; goto out; }
                net[v] += (w < 0 ? -w : 0) - (snk0 - sink[v]);
                value += snk0 - sink[v];
                if (z >= 2) {
                    if (fdown[v] < 0) { rc = 10; goto out; }
                    net[v] -= fdown[v];
                    net[v - 1] += fdown[v];
                } else if (fdown[v] != 0) { rc = 10; goto out; }
                for (int d = 0; d < 4; ++d) {
                    const int64_t xq = x + DX[d], yq = y + DY[d];
                    const int in_grid = xq >= 0 && xq < X && yq >= 0 && yq < Y;
                    const int64_t fhv = fhard[d * N + v];
                    if (in_grid && z - delta >= 1) {
                        if (fhv < 0) { rc = 10; goto out; }
                        const int64_t head = idx3(Y, Z, xq, yq, z - delta);
                        net[v] -= fhv;
                        net[head] += fhv;
                    } else if (fhv != 0) { rc = 10; goto out; }
                    if (d & 1) { /* the d = 0 pair towards x+1 / y+1 */
                        const int64_t gv = gpair[(d >> 1) * N + v];
                        if (in_grid && k0 > 0) {
                            if (gv < -k0 || gv > k0) { rc = 10; goto out; }
                            net[v] -= gv;
                            net[idx3(Y, Z, xq, yq, z)] += gv;
                        } else if (gv != 0) { rc = 10; goto out; }
                    }
                    for (int64_t dd = 1; dd < delta; ++dd) {
                        const int64_t fl = flayer[((dd - 1) * 4 + d) * N + v];
                        if (in_grid && z - dd >= 1 && kcap[dd] > 0) {
                            if (fl < 0 || fl > kcap[dd]) { rc = 10; goto out; }
                            net[v] -= fl;
                            net[idx3(Y, Z, xq, yq, z - dd)] += fl;
                        } else if (fl != 0) { rc = 10; goto out; }
                    }
                }
            }
    for (int64_t v = 0; v < N; ++v) {
        if (v % Z == 0) continue;
        if (net[v] != excess[v] || excess[v] < 0) { rc = 11; goto out; }
    }
    if (value != flow) { rc = 12; goto out; }
    /* residual reach of the excess nodes (z >= 1 only; the bottom layer is the source) */
    int64_t qh = 0, qt = 0;
    for (int64_t v = 0; v < N; ++v)
        if (v % Z != 0 && excess[v] > 0) { seen[v] = 1; queue[qt++] = v; }
    while (qh < qt) {
        const int64_t u = queue[qh++];
        const int64_t z = u % Z, col = u / Z, x = col / Y, y = col % Y;
#define ORC_REACH(node)                                  \
    do {                                                 \
        const int64_t _n = (node);                       \
        if (!seen[_n]) { seen[_n] = 1; queue[qt++] = _n; } \
    } while (0)
        if (z >= 2) ORC_REACH(u - 1);                        /* down arc: infinite */
        if (z + 1 < Z && fdown[u + 1] > 0) ORC_REACH(u + 1); /* reverse of the down arc above */
        for (int d = 0; d < 4; ++d) {
            const int64_t xq = x + DX[d], yq = y + DY[d];
            if (xq < 0 || xq >= X || yq < 0 || yq >= Y) continue;
            if (z - delta >= 1) ORC_REACH(idx3(Y, Z, xq, yq, z - delta));
            if (z + delta < Z) {
                const int64_t wq = idx3(Y, Z, xq, yq, z + delta);
                if (fhard[(d ^ 1) * N + wq] > 0) ORC_REACH(wq);
            }
            if (k0 > 0) {
                const int64_t q = idx3(Y, Z, xq, yq, z);
                const int64_t gv = (d & 1) ? gpair[(d >> 1) * N + u] : -gpair[(d >> 1) * N + q];
                if (k0 - gv > 0) ORC_REACH(q); /* gv: net flow u -> q */
            }
            for (int64_t dd = 1; dd < delta; ++dd) {
                if (kcap[dd] <= 0) continue;
                if (z - dd >= 1 && kcap[dd] - flayer[((dd - 1) * 4 + d) * N + u] > 0)
                    ORC_REACH(idx3(Y, Z, xq, yq, z - dd));
                if (z + dd < Z) { /* reverse of the layer arc of (q, z+dd) into u */
                    const int64_t wq = idx3(Y, Z, xq, yq, z + dd);
                    if (flayer[((dd - 1) * 4 + (d ^ 1)) * N + wq] > 0) ORC_REACH(wq);
                }
            }
        }
#undef ORC_REACH
    }
    for (int64_t v = 0; v < N; ++v) {
        if (v % Z == 0) continue;
        if ((in_cut[v] != 0) != (seen[v] != 0)) { rc = 13; goto out; }
    }
    for (int64_t col = 0; col < (int64_t)X * Y; ++col) {
        int32_t top = 0;
        for (int64_t z = 1; z < Z; ++z)
            if (in_cut[col * Z + z]) top = (int32_t)z;
        if (heights[col] != top) { rc = 14; goto out; }
    }
    if (oracle_cut_capacity_convex(cost, X, Y, Z, delta, f, heights) != flow) rc = 15;
out:
    free(kcap);
    free(net);
    free(seen);
    free(queue);
    return rc;
}
