// thin_naive.cu -- the reference slice of the CUDA path: one launch per
// subfield phase, straight from global memory, in place.
//
// Phase g visits the interior points of parity 2(y&1)+(x&1) = g mod 4.  Such
// points are pairwise not 8-adjacent, so each thread can read its 3x3 window
// and lower its point (Sec. 2.2 lowering loop, Sec. 2.1 predicate) without
// racing any other thread of the launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "thin_common.cuh"
#include "thin_internal.h"

namespace thin {

struct NaiveState {
    unsigned long long lowered;
    long long last_change;
    int changed;  // some point was lowered since the last reset
    int pad;
};

__device__ const PointTable d_naive_table = kPointTable;
__device__ const PointTable d_naive_table48 = kPointTable48;

template <typename T>
__global__ void __launch_bounds__(256) k_naive_phase(T *img, int w, int h, size_t pitch, int px, int py,
                                                     uint32_t lam, int mode, long long g, NaiveState *st)
{
    __shared__ uint32_t tab[256];
    tab[threadIdx.x] = (mode & 4) ? d_naive_table48.v[threadIdx.x] : d_naive_table.v[threadIdx.x];
    __syncthreads();
    const int x = 2 * (blockIdx.x * blockDim.x + threadIdx.x) + px;
    const int y = 2 * blockIdx.y + py;
    int nl = 0;
    if (x >= 1 && x <= w - 2 && y >= 1 && y <= h - 2) {
        char *base = reinterpret_cast<char *>(img);
        const T *up = reinterpret_cast<const T *>(base + size_t(y - 1) * pitch);
        T *row = reinterpret_cast<T *>(base + size_t(y) * pitch);
        const T *dn = reinterpret_cast<const T *>(base + size_t(y + 1) * pitch);
        uint32_t nb[8] = {row[x + 1], up[x + 1], up[x], up[x - 1], row[x - 1], dn[x - 1], dn[x], dn[x + 1]};
        const uint32_t c = row[x];
        const uint32_t c2 = lower_point(c, nb, tab, lam, mode, nl);
        if (nl) row[x] = static_cast<T>(c2);
    }
    // one atomic per warp
    unsigned lane = threadIdx.x & 31;
    int sum = nl;
    for (int o = 16; o; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
    if (lane == 0 && sum) {
        atomicAdd(&st->lowered, (unsigned long long)sum);
        atomicMax(&st->last_change, g);
        st->changed = 1;
    }
}

int naive_run(const JobSpec &job, const thin_options &opt, cudaStream_t stream, thin_stats *out)
{
    NaiveState *d = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&d), sizeof(NaiveState), stream);
    if (e != cudaSuccess) return THIN_ERR_OOM;
    NaiveState init{};
    init.last_change = -1;
    e = cudaMemcpyAsync(d, &init, sizeof init, cudaMemcpyHostToDevice, stream);
    const int pts_x = (job.w + 1) / 2, pts_y = (job.h + 1) / 2;
    const dim3 block(256), grid((pts_x + 255) / 256, std::max(pts_y, 1));
    long long g = opt.start_phase, run = 0;
    int status = THIN_OK, converged = 0;
    long long rounds = 0;
    const int zero = 0;
    while (e == cudaSuccess) {
        bool capped = false;
        for (int r = 0; r < 4; ++r) {
            if (opt.max_phases >= 0 && run >= opt.max_phases) {
                capped = true;
                break;
            }
            const int p = int(g & 3);
            if (job.dtype == THIN_U8)
                k_naive_phase<uint8_t><<<grid, block, 0, stream>>>(static_cast<uint8_t *>(job.img), job.w, job.h,
                                                                   job.pitch, p & 1, p >> 1, job.lam, test_mode(opt) | (job.adj << 2), g, d);
            else
                k_naive_phase<uint16_t><<<grid, block, 0, stream>>>(static_cast<uint16_t *>(job.img), job.w, job.h,
                                                                    job.pitch, p & 1, p >> 1, job.lam, test_mode(opt) | (job.adj << 2), g, d);
            ++g;
            ++run;
        }
        if (capped) {
            status = THIN_ERR_NOT_CONVERGED;
            break;
        }
        ++rounds;
        int changed = 0;
        e = cudaMemcpyAsync(&changed, &d->changed, sizeof changed, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) break;
        if (!changed) {
            converged = 1;
            break;
        }
        e = cudaMemcpyAsync(&d->changed, &zero, sizeof zero, cudaMemcpyHostToDevice, stream);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    NaiveState fin{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&fin, d, sizeof fin, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    cudaFreeAsync(d, stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (out) {
        std::memset(out, 0, sizeof *out);
        out->status = status;
        out->converged = converged;
        out->phases = run;
        out->lowered = (int64_t)fin.lowered;
        out->last_change_phase = fin.last_change;
        out->end_phase = g;
        out->tiles_visited = 0;
        out->steps = rounds;
        // every interior point of the phase's parity is tested in every phase
        long long per[4] = {0, 0, 0, 0};
        for (int p = 0; p < 4; ++p) {
            const long long nx = (job.w - 2 - ((p & 1) ? 1 : 2)) / 2 + 1, ny = (job.h - 2 - ((p >> 1) ? 1 : 2)) / 2 + 1;
            per[p] = (nx > 0 && ny > 0) ? nx * ny : 0;
        }
        long long t = 0;
        for (long long q = opt.start_phase; q < g; ++q) t += per[q & 3];
        out->tested = t;
    }
    return status;
}

}  // namespace thin
