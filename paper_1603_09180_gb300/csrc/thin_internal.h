// thin_internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/thin.h"

namespace thin {

// Validated description of one image handed to an engine.
struct JobSpec {
    void *img;
    int w, h;
    size_t pitch;
    int dtype;      // THIN_U8 / THIN_U16
    uint32_t lam;
};

inline int elem_size(int dtype) { return dtype == THIN_U16 ? 2 : 1; }

// Naive engine: one launch per subfield phase over the whole image, in place.
int naive_run(const JobSpec &job, const thin_options &opt, cudaStream_t stream, thin_stats *out);

// Tiled engine: TMA-staged tiles, temporal blocking, active-tile worklist,
// one persistent cooperative launch for any number of images.
int tiled_run(const JobSpec *jobs, int n, const thin_options &opt, cudaStream_t stream, thin_stats *out);

// Resident engine: each image held in the shared memory of one thread-block
// cluster of C blocks (1, 2, 4 or 8) of nw warps (4, 8 or 16; 16 / nw blocks
// share an SM) for its whole run.
int resident_run(const JobSpec *jobs, int n, int C, int nw, const thin_options &opt, cudaStream_t stream,
                 thin_stats *out);
// Smallest cluster of nw-warp blocks whose shared memory holds a w x h image
// of `dtype`, 0 if none.
int resident_cluster_size(int w, int h, int dtype, size_t smem_limit, int nw, int *rows_out, int *rp_out);
// Shared memory one block may take when `blocks` blocks share an SM.
size_t resident_smem_limit(int blocks);

// Defaults of the tiled engine for a dtype (tile width/height in pixels, halo).
void tiled_defaults(int dtype, int *tw, int *th, int *halo);

int cuda_status(cudaError_t e);

}  // namespace thin
