// thin_tune.cu -- the tiled engine's autotuner: tile shape and halo depth
// (phases per tile visit) picked by timing candidates on the image itself.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "thin_internal.h"

namespace thin {
namespace {

struct Candidate {
    int tw, th, halo;
};

// Tile shapes and halo depths the tiled engine accepts for both dtypes
// (tile width a multiple of 16 up to 224, even height, halo <= 8 and below
// the shorter tile side, tile height + 2 halo rows <= 256).
const Candidate kCandidates[] = {
    {64, 32, 8}, {64, 32, 6}, {64, 32, 4}, {128, 32, 8}, {64, 64, 8}, {128, 64, 8},
    {32, 32, 8}, {96, 48, 8}, {128, 16, 8}, {224, 32, 8}, {48, 64, 8}, {64, 16, 6},
};

}  // namespace
}  // namespace thin

using namespace thin;

extern "C" int thin_autotune(const void *img_dev, int w, int h, size_t pitch_bytes, thin_dtype dt, uint32_t lambda,
                             void *stream, int64_t trial_phases, thin_options *opt, float *best_ms)
{
    NvtxRange nv("thin_autotune");
    if (!opt) return THIN_ERR_ARG;
    if (w < 3 || h < 3 || !img_dev || (dt != THIN_U8 && dt != THIN_U16)) return THIN_ERR_ARG;
    const size_t es = elem_size(dt);
    if (pitch_bytes < size_t(w) * es) return THIN_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    thin_options base = *opt;
    base.kernel = THIN_KERNEL_TILED;
    base.max_phases = trial_phases;
    // the trials thin a scratch copy (16-byte aligned rows, as the engine likes them)
    const size_t sp = (size_t(w) * es + 127) / 128 * 128;
    void *scratch = nullptr;
    cudaError_t e = cudaMallocAsync(&scratch, sp * h, s);
    if (e != cudaSuccess) return cuda_status(e);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = -1.f;
    Candidate pick = {0, 0, 0};
    for (const Candidate &c : kCandidates) {
        if (e != cudaSuccess) break;
        thin_options o = base;
        o.tile_w = c.tw;
        o.tile_h = c.th;
        o.halo = c.halo;
        float ms = 0.f;
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first run warms the caches up
            e = cudaMemcpy2DAsync(scratch, sp, img_dev, pitch_bytes, size_t(w) * es, h, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) e = cudaEventRecord(e0, s);
            JobSpec j{scratch, w, h, sp, int(dt), lambda, THIN_ADJ_8_4};
            const int rc = e == cudaSuccess ? tiled_run(&j, 1, o, s, nullptr) : THIN_ERR_CUDA;
            if (rc == THIN_ERR_ARG) break;  // a shape this image's dtype does not take
            if (rc != THIN_OK && rc != THIN_ERR_NOT_CONVERGED) e = cudaErrorUnknown;
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (rep == 1 && e == cudaSuccess && (best < 0.f || ms < best)) {
                best = ms;
                pick = c;
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(scratch, s);
    if (e != cudaSuccess) return cuda_status(e);
    if (best < 0.f) return THIN_ERR_ARG;
    opt->tile_w = pick.tw;
    opt->tile_h = pick.th;
    opt->halo = pick.halo;
    if (best_ms) *best_ms = best;
    return THIN_OK;
}
