// Narrow-band construction of the proper-order graph around landmark points (Section 3.4:
// the user picks landmark points on a horizon; the structured graph spans, in every
// column, the stick length above and below a surface through those points, widened by
// the narrow-band factor). Two kernels, both bound by memory bandwidth:
//   k_band_center: one thread per column interpolates the landmark heights by inverse
//     squared distance (fp64, explicitly rounded operations in a fixed order, so the
//     result is reproducible bit for bit);
//   k_band_gather: one thread per band node copies the image cost at the column's
//     center - half + k (coalesced along the band rows), or the outside cost.
// A surface solved on the band maps back to image heights by adding center - half.
#include "pog.h"
#include "pog_internal.cuh"

namespace {

constexpr int kThreads = 256;

__global__ void k_band_center(const int32_t *lm, int L, int X, int Y, int Zi, int32_t *center) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= X * Y) return;
    const int x = col / Y, y = col - x * Y;
    double num = 0.0, den = 0.0;
    int on = -1;  // height of the first landmark on this column, if any
    for (int i = 0; i < L; ++i) {
        const int lx = __ldg(lm + 3 * i), ly = __ldg(lm + 3 * i + 1), lz = __ldg(lm + 3 * i + 2);
        const long long d2 = (long long)(x - lx) * (x - lx) + (long long)(y - ly) * (y - ly);
        if (d2 == 0) {
            if (on < 0) on = lz;
            continue;
        }
        const double w = __ddiv_rn(1.0, (double)d2);
        num = __dadd_rn(num, __dmul_rn(w, (double)lz));
        den = __dadd_rn(den, w);
    }
    int c = on;
    if (c < 0) c = (int)floor(__dadd_rn(__ddiv_rn(num, den), 0.5));  // round half up
    center[col] = c < 0 ? 0 : (c >= Zi ? Zi - 1 : c);
}

__global__ void k_band_gather(const int32_t *cost, const int32_t *center, int X, int Y, int Zi, int Zb, int half,
                              int outside, int32_t *band) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = (long long)X * Y * Zb;
    if (i >= n) return;
    const long long col = i / Zb;
    const int k = (int)(i - col * Zb);
    const int z = __ldg(center + col) - half + k;
    band[i] = (z >= 0 && z < Zi) ? __ldg(cost + col * Zi + z) : outside;
}

__global__ void k_band_heights(const int32_t *hb, const int32_t *center, int cols, int half, int32_t *himg) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col < cols) himg[col] = center[col] - half + hb[col];
}

int blocks_for(long long n) { return (int)((n + kThreads - 1) / kThreads); }

pog_status status_of(cudaError_t e) {
    return e == cudaSuccess ? POG_OK : (e == cudaErrorMemoryAllocation ? POG_E_NOMEM : POG_E_CUDA);
}

}  // namespace

extern "C" {

pog_status pog_narrow_band(const int32_t *cost_dev, int32_t X, int32_t Y, int32_t Zi, const int32_t *landmarks_dev,
                           int32_t L, int32_t stick, int32_t band_factor, int32_t outside_cost, void *stream,
                           int32_t *band_dev, int32_t *center_dev) {
    if (!cost_dev || !landmarks_dev || !band_dev || !center_dev || X < 1 || Y < 1 || Zi < 1 || L < 1 ||
        stick < 0 || band_factor < 1 || outside_cost <= -(1 << 30) || outside_cost >= (1 << 30))
        return POG_E_INVALID;
    const long long half = (long long)stick * band_factor;
    const long long Zb = 2 * half + 1;
    if (Zb >= (1 << 30) || (long long)X * Y * Zb >= (1ll << 31) - 64) return POG_E_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_band_center<<<blocks_for((long long)X * Y), kThreads, 0, st>>>(landmarks_dev, L, X, Y, Zi, center_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return status_of(e);
    k_band_gather<<<blocks_for((long long)X * Y * Zb), kThreads, 0, st>>>(cost_dev, center_dev, X, Y, Zi, (int)Zb,
                                                                          (int)half, outside_cost, band_dev);
    return status_of(cudaGetLastError());
}

pog_status pog_band_heights(const int32_t *h_band_dev, const int32_t *center_dev, int32_t X, int32_t Y, int32_t half,
                            void *stream, int32_t *h_img_dev) {
    if (!h_band_dev || !center_dev || !h_img_dev || X < 1 || Y < 1 || half < 0) return POG_E_INVALID;
    k_band_heights<<<blocks_for((long long)X * Y), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        h_band_dev, center_dev, X * Y, half, h_img_dev);
    return status_of(cudaGetLastError());
}

}  // extern "C"
