/*
 * pog.h — C ABI of the GB300 min-cut solver for proper-order multi-column graphs.
 *
 * The problem (Section 1.2 and Section 1.3 of Chandramouli, "Parallel Algorithm For
 * Finding The Minimum s-t Cut in a Structured 3-Dimensional Proper Order Graph"):
 * a cost volume c(x, y, z) over X*Y columns of Z nodes defines the surface energy of
 * Eq. 1,
 *     E(h) = sum_col c(col, h(col)) + alpha * sum_{4-neighbour pairs} |h_p - h_q|,
 * subject to |h_p - h_q| <= delta. Its minimiser is the source side of the minimum
 * s-t cut (Theorem 1.1) of the proper-order graph whose node weights
 * w(z) = c(z) - c(z-1) become terminal arcs. The library computes the maximum flow
 * value (Eq. 5) and the surface of the minimal minimum cut (the nodes reachable from
 * s in the final residual graph), whose height in each column is the top node of the
 * cut there. Vertices and arcs are addressed implicitly from (x, y, z) (Section 3.2.3);
 * no edge list exists anywhere.
 *
 * Layout: every volume is int32 (or float32) [X][Y][Z], z fastest: element (x, y, z)
 * at ((x*Y + y)*Z + z) — a contiguous torch tensor of shape [X, Y, Z]. A height map is
 * int32 [X][Y], column (x, y) at x*Y + y.
 *
 * Pointers: "device" pointers are CUDA global-memory addresses on the current device;
 * "host" pointers are ordinary CPU memory. The caller owns every pointer it passes;
 * the library never keeps one past the call (pog_build copies what it needs into its
 * own state before its stream work completes) and never frees one.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 * stream). All device work of a graph is ordered on the stream given to pog_build.
 *
 * Errors: every call returns a pog_status. No call throws, traps, or aborts; device
 * failures are reported through a device error word read back by the host. After an
 * error other than POG_E_INVALID the graph may only be freed.
 */
#ifndef POG_H
#define POG_H

#include <stdint.h>

#if defined(__GNUC__)
#define POG_API __attribute__((visibility("default")))
#else
#define POG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    POG_OK = 0,
    POG_E_INVALID = 1,    /* bad argument: sizes < 1, delta/alpha < 0, NULL pointer, N too large */
    POG_E_OVERFLOW = 2,   /* a cost with |c| >= 2^30, or an arc flow that reached the int32 range */
    POG_E_NOMEM = 3,      /* device or pinned-host allocation failed */
    POG_E_CUDA = 4,       /* a CUDA runtime call failed (launch, copy, sync) */
    POG_E_NOCONVERGE = 5, /* the iteration cap of pog_options was reached */
    POG_E_TIMEOUT = 6,    /* a bounded device-side wait gave up */
    POG_E_STATE = 7       /* call out of order, e.g. pog_surface before pog_maxflow */
} pog_status;

/* Tuning knobs. Zero in a field selects the built-in default. */
typedef struct {
    int32_t sweeps_per_relabel; /* push/relabel sweeps between global relabels (Section 2.1) */
    int32_t max_rounds;         /* cap on global-relabel rounds before POG_E_NOCONVERGE */
    int32_t tile_sweeps;        /* local push/relabel sweeps per shared-memory tile visit */
    int32_t flags;              /* POG_FLAG_* bits */
    int32_t bfs_blocks_per_sm;  /* blocks per SM of the cooperative BFS launches: 1, 2 or 4 (of 1024,
                                   512 or 256 threads); 0 or other values: 4 */
    float relabel_factor;       /* adaptive mode: sweep time per round / global relabel time */
    int32_t tile_shape;         /* 0: 4x8 columns x 32 heights, 1: 8x8x16, 2: 4x4x64, 3: 2x4x128 */
    int32_t bfs_bottom_up_ratio; /* BFS level runs bottom-up when frontier * ratio > unlabelled
                                    nodes; 0 = default (8), < 0 = always top-down */
    /* Test hooks for the failure paths (leave 0 in production): */
    int32_t test_wait_limit;    /* polls of the searches' grid-barrier wait before it gives up and
                                   the call returns POG_E_TIMEOUT; 0 = the built-in limit */
    int32_t test_fail_alloc;    /* k > 0: the k-th allocation of a graph build (1 device state,
                                   2 tensor-map table, 3 pinned counters) fails as if memory had
                                   run out (POG_E_NOMEM, nothing kept) */
} pog_options;

#define POG_FLAG_NO_GAP 1     /* disable the gap heuristic between global relabels */
#define POG_FLAG_TIMING 2     /* time each kernel family with CUDA events on the graph's stream */
#define POG_FLAG_NO_PREPUSH 4 /* skip the column pre-push along the down arcs */
#define POG_FLAG_NODE_SWEEPS 8 /* node-parallel sweeps instead of shared-memory tiles */
#define POG_FLAG_NO_TMA 16    /* load shared-memory tiles word by word, not by bulk tensor copies */
#define POG_FLAG_COLD_HINGE 32 /* pog_solve_batch_f32_hinge: solve the loss-augmented problem from
                                  scratch instead of from the energy solve's final state */

/* Counters of the last pog_maxflow. */
typedef struct {
    int64_t rounds;          /* global relabels run (the initial one included) */
    int64_t sweeps;          /* push/relabel sweep launches */
    int64_t bfs_passes;      /* global-relabel relaxation passes */
    int64_t cut_passes;      /* cut-extraction reachability passes */
    int64_t gaps;            /* gap relabels that raised at least one label */
    int64_t active_initial;  /* active nodes after the initial global relabel */
    int64_t nodes;           /* X*Y*Z */
    int64_t state_bytes;     /* device bytes of the residual state */
    int64_t launches;        /* kernels launched by pog_build + pog_maxflow */
    int64_t tiles_visited;   /* tiles staged in shared memory by the tiled sweeps */
    /* device milliseconds per kernel family, with POG_FLAG_TIMING only (else 0) */
    double sweep_ms;         /* push/relabel sweeps */
    double bfs_ms;           /* global-relabel relaxation passes */
    double cut_ms;           /* cut-extraction passes */
    double build_ms;         /* graph construction (pog_build) */
} pog_stats_t;

typedef struct pog_graph pog_graph; /* opaque; owns its device state */

/*
 * Build the residual graph of one volume (graph construction, Section 1.2; implicit
 * addressing, Section 3.2.3) and initialise the preflow: node weights become source
 * excess (w < 0) or sink residual (w > 0), all arc flows start at zero.
 *   cost_dev : device, int32 [X][Y][Z], |c| < 2^30 (else POG_E_OVERFLOW from pog_maxflow).
 *   X, Y, Z  : >= 1, X*Y*Z < 2^31.
 *   delta    : hard smoothness, >= 0 (|h_p - h_q| <= delta).
 *   alpha    : soft smoothness per unit height difference, 0 <= alpha < 2^30.
 *   opt      : host, may be NULL (defaults).
 *   stream   : cudaStream_t for all device work of this graph.
 *   out      : host, receives the new graph; unchanged on error.
 * Allocates about 48 bytes per node on the device (40 when alpha == 0): the residual
 * state and two search queues, plus a few small tables. Work is enqueued on `stream`;
 * `cost_dev` must stay valid until that work has run.
 */
POG_API pog_status pog_build(const int32_t *cost_dev, int32_t X, int32_t Y, int32_t Z, int32_t delta,
                     int32_t alpha, const pog_options *opt, void *stream, pog_graph **out);

/*
 * As pog_build, from a float32 device volume quantised on the fly to
 * cq = round_half_even(scale * c) (scale a power of two keeps the product exact).
 * A value with |scale * c| >= 2^30 or not finite makes pog_maxflow return POG_E_OVERFLOW.
 */
POG_API pog_status pog_build_f32(const float *cost_dev, float scale, int32_t X, int32_t Y, int32_t Z,
                         int32_t delta, int32_t alpha, const pog_options *opt, void *stream,
                         pog_graph **out);

/*
 * As pog_build_f32, with `margin` added to the quantised cost of the node (x, y, h(x,y))
 * of every column, where h_aug_dev is a device int32 [X][Y] surface. This builds the
 * loss-augmented problem min_h [E(h) - margin * Hamming(h, h_aug)] (up to the constant
 * margin * X * Y) of a structured hinge loss. 0 <= margin < 2^28.
 */
POG_API pog_status pog_build_f32_augmented(const float *cost_dev, float scale, const int32_t *h_aug_dev,
                                           int32_t margin, int32_t X, int32_t Y, int32_t Z, int32_t delta,
                                           int32_t alpha, const pog_options *opt, void *stream,
                                           pog_graph **out);

/*
 * Run push-relabel (Section 2.1; Algorithm 2) with periodic global relabelling by a
 * level-synchronous reverse BFS from the sink (Section 3.2.2; Algorithm 3), the gap
 * heuristic, and an exact termination test (Section 3.2.4) to a maximum preflow; then
 * extract the minimal minimum cut and the surface heights.
 *   flow_out : host, receives the max-flow value (int64) of the literal s-t graph.
 * Blocks the calling thread until the graph's stream has finished this work.
 */
POG_API pog_status pog_maxflow(pog_graph *g, int64_t *flow_out);

/*
 * Copy the surface heights of the last pog_maxflow.
 *   heights_dev : device, int32 [X][Y], receives h(x, y) in [0, Z).
 * Enqueued on the graph's stream (asynchronous). POG_E_STATE before pog_maxflow.
 */
POG_API pog_status pog_surface(pog_graph *g, int32_t *heights_dev);

/*
 * Optimal energy E*(h) of Eq. 1 (in the units of the built costs) of the last
 * pog_maxflow, from the flow value: max-flow = E*(h) + K, where
 * K = -1 - sum_col c(col, 0) + sum over nodes with w < 0 of -w (the cut capacity of
 * Eq. 6 for the closed set below h, after the weights telescope along each column).
 *   energy_out : host int64.
 */
POG_API pog_status pog_energy(const pog_graph *g, int64_t *energy_out);

/*
 * Energy of Eq. 1 of given surfaces on quantised float costs, one volume per entry:
 *   energy[b] = sum_col round_half_even(scale * c[b][col][h]) + alpha * sum_pairs |h_p - h_q|.
 * Device pointers: cost float32 [B][X][Y][Z], h int32 [B][X][Y], energy int64 [B].
 * A height outside [0, Z) makes that volume's entry INT64_MIN. Enqueued on `stream`.
 */
POG_API pog_status pog_surface_energy(const float *cost_dev, float scale, const int32_t *h_dev, int32_t B,
                                      int32_t X, int32_t Y, int32_t Z, int32_t alpha, int64_t *energy_dev,
                                      void *stream);

/* Counters of the last pog_maxflow. out: host. */
POG_API pog_status pog_stats(const pog_graph *g, pog_stats_t *out);

/*
 * Diagnostics: the per-level trace of the last global relabel (reverse BFS, Algorithm 3).
 *   out        : host int64 [3 * max_levels]; entry i holds (frontier size, mode, device
 *                time in ns) of level i+1, mode 0 = top-down queue expansion, 1 =
 *                bottom-up scan; the final entry has mode -1 and marks the end time.
 *   levels_out : host, receives the number of entries written (0 if more than
 *                min(max_levels, 4096) levels ran).
 * Synchronises the graph's stream.
 */
POG_API pog_status pog_trace(const pog_graph *g, int64_t *out, int32_t max_levels, int32_t *levels_out);

/*
 * Download the residual state after pog_maxflow, for host-side certificates.
 * Each pointer is host memory of N = X*Y*Z int32 (fh: 4*N, gs: 2*N when alpha > 0,
 * else may be NULL); any may be NULL to skip it. Node (x,y,z) at ((x*Y+y)*Z+z).
 *   excess : final excess of each node (z >= 1; z = 0 nodes report 0).
 *   sink   : remaining residual capacity of the node's arc to the sink.
 *   fdown  : flow on the infinite arc (x,y,z) -> (x,y,z-1), z >= 2.
 *   fhard  : fhard[d*N + v]: flow on the infinite arc from v to its neighbour in
 *            direction d (0: x-1, 1: x+1, 2: y-1, 3: y+1) at height z - delta
 *            (present when z - delta >= 1).
 *   gsoft  : gsoft[k*N + v]: net flow from v to its neighbour at x+1 (k = 0) or
 *            y+1 (k = 1) at the same z, in [-alpha, alpha].
 *   in_cut : 1 when the node is in the source side of the minimal minimum cut.
 * Arcs into the bottom layer z = 0 carry no flow here: the bottom layer is always in
 * the minimal cut, so the solver merges it into the source (its sink arcs add a
 * constant to the flow value).
 */
POG_API pog_status pog_export_state(const pog_graph *g, int32_t *excess, int32_t *sink, int32_t *fdown,
                            int32_t *fhard, int32_t *gsoft, int32_t *in_cut);

/* Release the graph and its device state (synchronises its stream first). NULL is a no-op. */
POG_API void pog_free(pog_graph *g);

/* Static, human-readable text of a status. */
POG_API const char *pog_strerror(pog_status s);

/*
 * Quantise a float32 device array to int32: out[i] = round_half_even(scale * in[i]).
 * Same rule as pog_build_f32. Returns POG_E_OVERFLOW (after a stream sync) when some
 * |scale * in[i]| >= 2^30 or is not finite.
 */
POG_API pog_status pog_quantise(const float *in_dev, int32_t *out_dev, int64_t n, float scale,
                        void *stream);

/*
 * Backward of the optimal energy E*(c) = min_h E(h) with respect to the cost volume
 * (Danskin's theorem: the one-hot of the optimal surface), combined with a second
 * surface for the structured hinge loss:
 *   grad[b][x][y][z] = g_energy[b] * [z == h[b][x][y]]
 *                    + g_hinge[b]  * ([z == h_target[b][x][y]] - [z == h_hat[b][x][y]])
 * Device pointers: grad float32 [B][X][Y][Z] (fully overwritten), h / h_target / h_hat
 * int32 [B][X][Y] (h_target and h_hat may be NULL when g_hinge is NULL), g_energy and
 * g_hinge float32 [B] (device; g_hinge may be NULL). Enqueued on `stream`.
 */
POG_API pog_status pog_backward(float *grad_dev, const int32_t *h_dev, const int32_t *h_target_dev,
                        const int32_t *h_hat_dev, const float *g_energy_dev,
                        const float *g_hinge_dev, int32_t B, int32_t X, int32_t Y, int32_t Z,
                        void *stream);

/* One volume of a batch: device cost pointer, sizes and smoothness. */
typedef struct {
    const int32_t *cost_dev;
    int32_t X, Y, Z, delta, alpha;
} pog_volume;

/*
 * Solve n independent volumes (sizes may differ) as one batch: the disjoint union of
 * their graphs goes through the same launches (one global relabel, one tiled sweep, one
 * cut extraction for all of them), and volumes leave the work once their relabel finds
 * no active node. flows_out: host int64 [n]; heights_dev[i]: device int32 [X_i][Y_i].
 * Blocks until done. At most 1024 volumes, fewer than 2^31 nodes in all.
 */
POG_API pog_status pog_solve_batch(int32_t n, const pog_volume *vols, const pog_options *opt,
                           void *stream, int64_t *flows_out, int32_t *const *heights_dev);

/*
 * Solve B float32 volumes of one shape as one batch (the differentiable path): each is
 * quantised on the fly to round_half_even(scale * c), optionally with `margin` added at
 * node (x, y, h_aug[b][x][y]) as in pog_build_f32_augmented.
 *   cost_dev     : device float32 [B][X][Y][Z].
 *   h_aug_dev    : device int32 [B][X][Y], or NULL for no augmentation.
 *   flows_out    : host int64 [B], max-flow values.
 *   energies_out : host int64 [B] or NULL, optimal energies E*(h) (as pog_energy).
 *   heights_dev  : device int32 [B][X][Y], the surfaces.
 * Blocks until done.
 */
POG_API pog_status pog_solve_batch_f32(int32_t B, const float *cost_dev, float scale, const int32_t *h_aug_dev,
                                       int32_t margin, int32_t X, int32_t Y, int32_t Z, int32_t delta,
                                       int32_t alpha, const pog_options *opt, void *stream, int64_t *flows_out,
                                       int64_t *energies_out, int32_t *heights_dev);

/*
 * Structured-hinge forward of B float32 volumes of one shape in one call: the energy
 * solve, the loss-augmented solve and the loss (the differentiable path). Each volume is
 * quantised to cq = round_half_even(scale * c) as in pog_solve_batch_f32, then
 *   E*     = min_h E(h) (Eq. 1 on cq), with its minimal surface h*;
 *   E'*    = min_h E'(h), E' the energy of the costs with `margin` added at node
 *            (x, y, h_t(x, y)) of every column, with its minimal surface h_hat; so
 *            min_h [E(h) - margin * Hamming(h, h_t)] = E'* - margin * X * Y;
 *   L      = E(h_t) - (E'* - margin * X * Y), the structured hinge loss (>= 0 when h_t is
 *            feasible), whose subgradient in the costs is onehot(h_t) - onehot(h_hat).
 * The loss-augmented problem is solved from the final residual state of the energy solve
 * (its costs differ at one node per column, and the state becomes a preflow of it by
 * raising two terminal capacities per column), unless POG_FLAG_COLD_HINGE is set.
 *   cost_dev       : device float32 [B][X][Y][Z].
 *   h_target_dev   : device int32 [B][X][Y], heights in [0, Z) (else POG_E_INVALID).
 *   margin         : 0 <= margin < 2^28, in quantised units.
 *   energies_out   : host int64 [B], E*.
 *   aug_energies_out : host int64 [B] or NULL, E'*.
 *   hinge_out      : host int64 [B], L in quantised units.
 *   flows_out, aug_flows_out : host int64 [B] or NULL, the max-flow values of the two
 *                    problems' graphs (Section 1.2 construction).
 *   heights_dev, h_hat_dev : device int32 [B][X][Y], h* and h_hat.
 * Blocks until done.
 */
POG_API pog_status pog_solve_batch_f32_hinge(int32_t B, const float *cost_dev, float scale,
                                             const int32_t *h_target_dev, int32_t margin, int32_t X, int32_t Y,
                                             int32_t Z, int32_t delta, int32_t alpha, const pog_options *opt,
                                             void *stream, int64_t *energies_out, int64_t *aug_energies_out,
                                             int64_t *hinge_out, int64_t *flows_out, int64_t *aug_flows_out,
                                             int32_t *heights_dev, int32_t *h_hat_dev);

/*
 * Narrow-band construction (Section 3.4): the structured graph built around landmark
 * points on a horizon. In each column it spans `half` = stick * band_factor rows below
 * and above a center surface through the landmarks, Zb = 2 * half + 1 rows in all.
 * The paper gives no formula for that surface; here it is the inverse-squared-distance
 * average of the landmark heights, rounded half up:
 *   center(x, y) = floor(sum_i w_i z_i / sum_i w_i + 0.5),  w_i = 1 / ((x-x_i)^2 + (y-y_i)^2),
 * in float64 with every operation rounded to nearest, summed in landmark order (the
 * height z_i of the first landmark on the column itself when there is one), clamped to
 * [0, Zi). The band cost volume is
 *   band(x, y, k) = cost(x, y, center - half + k)   if 0 <= center - half + k < Zi,
 *                   outside_cost                     otherwise,
 * a volume of X * Y * Zb nodes for pog_build / pog_solve_noalloc; its surface maps back to
 * image heights with pog_band_heights.
 *   cost_dev      : device int32 [X][Y][Zi], the image cost volume.
 *   landmarks_dev : device int32 [L][3], (x, y, z) of each landmark, 0 <= z < Zi; L >= 1.
 *   stick, band_factor : >= 0 and >= 1; X * Y * Zb < 2^31.
 *   outside_cost  : |outside_cost| < 2^30, the cost of rows outside the image.
 *   band_dev      : device int32 [X][Y][Zb] (out).   center_dev : device int32 [X][Y] (out).
 * Enqueued on `stream`.
 */
POG_API pog_status pog_narrow_band(const int32_t *cost_dev, int32_t X, int32_t Y, int32_t Zi,
                                   const int32_t *landmarks_dev, int32_t L, int32_t stick, int32_t band_factor,
                                   int32_t outside_cost, void *stream, int32_t *band_dev, int32_t *center_dev);

/*
 * Image heights of a surface solved on a narrow band: h_img = center - half + h_band.
 * Device int32 [X][Y] each. Enqueued on `stream`.
 */
POG_API pog_status pog_band_heights(const int32_t *h_band_dev, const int32_t *center_dev, int32_t X, int32_t Y,
                                    int32_t half, void *stream, int32_t *h_img_dev);

/*
 * Solve one volume without allocating anything (the paper has no counterpart; this
 * entry point exists for callers of this library, not for the method).
 *
 * Who needs it: code that may not call cudaMalloc or any other allocating routine.
 * Examples are a host framework that owns every byte of device memory through its own
 * pool and forbids libraries from allocating behind its back, and latency-bound loops
 * in which cudaMalloc's implicit device-wide synchronisation cannot be afforded.
 * pog_build allocates its state with cudaMalloc (and pinned host memory and events);
 * this call instead does the whole solve (what pog_build, pog_maxflow and pog_surface
 * do together) with every scratch word in one fixed device array that the library
 * defines at file scope, POG_NOALLOC_SCRATCH_BYTES (32 MiB) in size. Every GPU on which
 * the library is loaded holds that array until the process exits.
 *
 * Limit: the volume's scratch must fit the array. It needs 48 bytes per node with
 * alpha > 0 (40 with alpha == 0) plus about 130 KiB, so about 690,000 nodes with a soft
 * penalty or 830,000 without. Larger volumes return POG_E_INVALID; use pog_build.
 *
 *   cost_dev    : device, int32 [X][Y][Z], as for pog_build.
 *   X, Y, Z, delta, alpha, opt : as for pog_build. sweeps_per_relabel is fixed here
 *                 (default 64): this path keeps no timing events, so the adaptive
 *                 choice is off. POG_FLAG_TIMING and the relabel trace are ignored.
 *   stream      : cudaStream_t for all device work.
 *   flow_out    : host, receives the max-flow value.
 *   heights_dev : device, int32 [X][Y], receives the surface heights (caller-owned).
 * Blocks until the stream has finished the solve. Allocates no device or host memory,
 * creates no events and calls no allocating library routine.
 *
 * Set-up: every call looks up the array's device address with cudaGetSymbolAddress
 * (with the device current), so no address outlives the context it came from. The first
 * call on a device also loads the library's device code there, which places the array
 * in that device's memory; make that first call before any stream capture begins on the
 * device.
 *
 * Sharing: every call on a device uses the same array, which keeps the last call's
 * contents (each call clears what must start at zero). Calls whose device work
 * overlaps — on two streams, or from two host threads — race on the array and give
 * wrong results; serialise them.
 */
#define POG_NOALLOC_SCRATCH_BYTES (32u << 20)
POG_API pog_status pog_solve_noalloc(const int32_t *cost_dev, int32_t X, int32_t Y, int32_t Z, int32_t delta,
                                     int32_t alpha, const pog_options *opt, void *stream, int64_t *flow_out,
                                     int32_t *heights_dev);

/*
 * Convex pairwise costs: the general optimal VCE-weight net surface of Section 1.2, whose
 * proper-order graph joins every vertex to an interval of vertices of each adjacent
 * column, with convex costs over that edge interval. Minimises
 *     E(h) = sum_col c(col, h(col)) + sum_{4-neighbour pairs} f(|h_p - h_q|)
 * subject to |h_p - h_q| <= delta, for a convex f with f(0) = 0. The graph carries, besides
 * the column and hard arcs of pog_build, one layer of soft arcs (x,y,z) -> (x',y',z-d) per
 * height drop d = 0 .. delta-1, of capacity k_0 = f(1) and k_d = f(d+1) - 2 f(d) + f(d-1):
 * a surface cuts (h_p - h_q - d)^+ arcs of layer d from column p to column q, and
 * sum_d k_d (t - d)^+ = f(t). pog_build's alpha is the profile f(t) = alpha * t (layer 0
 * only). Solved on the device by push-relabel with global relabelling and the minimal
 * cut's reach, every arc addressed from (x, y, z) as in pog_build.
 *   cost_dev    : device, int32 [X][Y][Z], |c| < 2^30 (else POG_E_OVERFLOW).
 *   X, Y, Z     : >= 1, X*Y*Z < 2^31.
 *   delta       : 0 <= delta <= POG_CONVEX_MAX_DELTA.
 *   f_host      : host, int64 [delta]: f(1), ..., f(delta) (may be NULL when delta = 0).
 *                 POG_E_INVALID unless 0 <= k_d < 2^30 for every d (f convex, f(1) >= 0).
 *   opt         : host, may be NULL. Used: sweeps_per_relabel (default 64), max_rounds,
 *                 flags (POG_FLAG_TIMING), test_fail_alloc (1: the state allocation fails).
 *   stream      : cudaStream_t for all device work.
 *   flow_out    : host, receives the max-flow value of the literal s-t graph.
 *   energy_out  : host, may be NULL: receives E*(h) = max-flow - K (K as for pog_energy).
 *   heights_dev : device, int32 [X][Y]: the surface of the minimal minimum cut.
 *   stats_out   : host, may be NULL: counters of this solve (pog_stats_t); this path has no
 *                 tiles, and its tiles_visited field counts the active nodes listed for the
 *                 push/relabel sweeps, summed over the sweeps. Also filled when the call
 *                 returns POG_E_NOCONVERGE (the counters up to the round cap).
 * Allocates (10 + 4 L) * 4 + 12 bytes per node on the device (L = layers d >= 1 with
 * k_d > 0) and frees them before returning; blocks until the work on `stream` is done.
 */
#define POG_CONVEX_MAX_DELTA 32
POG_API pog_status pog_solve_convex(const int32_t *cost_dev, int32_t X, int32_t Y, int32_t Z, int32_t delta,
                                    const int64_t *f_host, const pog_options *opt, void *stream,
                                    int64_t *flow_out, int64_t *energy_out, int32_t *heights_dev,
                                    pog_stats_t *stats_out);

#ifdef __cplusplus
}
#endif

#endif /* POG_H */
