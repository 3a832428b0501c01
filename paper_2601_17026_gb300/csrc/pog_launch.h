// Host-side launchers of the solver's kernels (all enqueue on the given stream and
// return the launch status).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pog {

struct Grid;
struct Batch;
struct BfsSync;

cudaError_t launch_build_i32(const Grid &g, const int32_t *cost, cudaStream_t st);
cudaError_t launch_build_f32(const Grid &g, const float *cost, float scale, const int32_t *h_aug, int margin,
                             cudaStream_t st);
cudaError_t launch_column_prepush(const Grid &g, cudaStream_t st);
// Turn the final state of a plain float-cost solve into a preflow of its loss-augmented
// problem (margin added at node (x, y, ht(x, y)) of every column); see k_augment.
cudaError_t launch_augment(const Grid &g, const float *cost, float scale, const int32_t *ht, int margin,
                           cudaStream_t st);
cudaError_t launch_sweep(const Batch &b, int *list, int *count, int ops, cudaStream_t st);
cudaError_t launch_gap(const Batch &b, unsigned int *bits, int levels, cudaStream_t st);
cudaError_t launch_heights(const Grid &g, int32_t *heights, cudaStream_t st);
cudaError_t launch_excess_sum(const Grid &g, cudaStream_t st);
cudaError_t launch_quantise(const float *in, int32_t *out, long long n, float scale, int *err, cudaStream_t st);
cudaError_t launch_backward(float *grad, const int32_t *h, const int32_t *ht, const int32_t *hh, const float *ge,
                            const float *gh, int B, int XY, int Z, cudaStream_t st);
cudaError_t launch_global_relabel(const Batch &b, const Grid *single, int *qa, int *qb, BfsSync *sync,
                                  int blocks_per_sm, int bottom_up_ratio, cudaStream_t st);
cudaError_t launch_cut_reach(const Batch &b, const Grid *single, int *qa, int *qb, BfsSync *sync, int blocks_per_sm,
                             cudaStream_t st);
constexpr int kTileShapes = 4;
long long tile_count(const Grid &g, int shape);
long long tile_count_max(const Grid &g);
// Encode the tensor maps of a volume's tile arrays (kTileArrays x kTensorMapBytes bytes,
// host memory at `out`) for the boxes of tile shape `shape`; false when the volume cannot
// use bulk tensor copies (z extent not a multiple of 4, an unaligned array, no driver
// support), in which case the tile kernel loads words one by one.
bool encode_tile_maps(const Grid &g, int shape, void *out);
// `tiles`: 4 arrays of `ntiles` ints (flag and list of two alternating sweep lists, all
// flags zero at the start); `work`: 6 ints, zero at the start. `serial` counts the
// tiled sweeps run on these buffers; `full_scan` is set on the first sweep after each
// global relabel.
cudaError_t launch_tile_sweep(const Batch &b, const Grid *single, int single_tile_base, bool soft, int shape,
                              int *tiles, long long ntiles, int *work, long long serial, bool full_scan,
                              int local_sweeps, cudaStream_t st);
cudaError_t launch_surface_energy(const float *cost, float scale, const int32_t *h, int B, int X, int Y, int Z,
                                  int alpha, long long *out, cudaStream_t st);

}  // namespace pog
