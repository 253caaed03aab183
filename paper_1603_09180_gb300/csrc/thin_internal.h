// thin_internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/thin.h"

namespace thin {

// An NVTX range over a C-ABI call, for Nsight Systems timelines.  The NVTX
// header only forwards to a profiler that is attached; otherwise it costs a
// branch.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Validated description of one image handed to an engine.
struct JobSpec {
    void *img;
    int w, h;
    size_t pitch;
    int dtype;      // THIN_U8 / THIN_U16
    uint32_t lam;
    int adj;        // THIN_ADJ_8_4 / THIN_ADJ_4_8
    int done_slot = -1;  // resident engine: completion record to post when the image is finished, -1 none
};

inline int elem_size(int dtype) { return dtype == THIN_U16 ? 2 : 1; }

// The point test's mode word for the kernels: bit 0 the F^- reading
// (thin_rule), bit 1 the operator (thin_op); the kernels add bit 2, the
// image's adjacency pair (thin_adj).
inline int test_mode(const thin_options &o) { return (o.rule & 1) | ((o.op & 1) << 1); }

// Naive engine: one launch per subfield phase over the whole image, in place.
int naive_run(const JobSpec &job, const thin_options &opt, cudaStream_t stream, thin_stats *out);

// Tiled engine: TMA-staged tiles, temporal blocking, active-tile worklist,
// one persistent cooperative launch for any number of images.
int tiled_run(const JobSpec *jobs, int n, const thin_options &opt, cudaStream_t stream, thin_stats *out);

// Resident engine: each image held in the shared memory of one thread-block
// cluster of C blocks (1, 2, 4 or 8) of 16 warps, one block per SM, for its
// whole run; one launch per cluster size and element size.
// Device-side records of the resident engine (thin_resident.cu).
struct ResJob {
    unsigned long long img;    // the caller's image, thinned in place
    unsigned long long pitch;  // bytes between rows
    int w, h, dtype;
    unsigned lam;
    int rows;   // image rows per block (even)
    int rp;     // shared row pitch in bytes: 16 B pad | w * es | pad to 16 | 16 B pad
    int cw;     // cells per row = ceil(w / 8)
    int wpr;    // bitmap words per cell row = ceil(cw / 32)
    int bulk;   // rows are 16-byte aligned and a multiple of 16 bytes: stage them by bulk copy
    int index;  // position of the job in the caller's list
    int hr;     // halo rows copied from each neighbouring block (even; 0 for a one-block cluster)
    int steph;  // phases between exchanges of halo rows
    int adj;    // thin_adj
    int done_slot;  // completion record of the job (ResArgs::done), -1 none
    unsigned long long ck;  // first word of the job's checkpoint of its dirty bitmaps (ResArgs::ckbits)
};

// Where a job paused at the end of its last time slice (ResArgs::slice).
struct ResRun {
    long long g;     // global phase index to resume at
    long long last;  // last phase that lowered a point, -1 if none
    int resumed;     // 1: the job has a checkpoint to resume from
    int pad;
};

struct ResStat {
    unsigned long long lowered;
    unsigned long long tested;   // point tests on own rows
    long long last_change;  // global phase index, -1 if none
    long long phases;
    int converged;
    int error;
};

// Completion record of one job, in host-mapped memory: the job's stats, then
// `flag` set to 1 (a system-scope release store) once its image is back in
// the caller's memory.  The host resets flag to 0 before the launch.
struct ResDone {
    ResStat st;
    int error;       // the launch's error word when the job finished
    unsigned flag;
};

struct ResCtl {
    unsigned head, tail;  // job ring: entries head .. tail - 1 wait to run (ResArgs::ring)
    int error;
    unsigned bar_count;  // grid barrier of a wide launch
    unsigned bar_gen;
    long long gl_last;   // wide launch: last phase that lowered a point anywhere, -1 if none
};

struct ResArgs {
    const ResJob *jobs;
    ResStat *st;
    ResCtl *ctl;
    int njobs;
    int rule;
    long long start_phase;
    long long max_phases;
    unsigned long long timeout_ns;
    // Wide launch (strips > 0): one image over `strips` clusters, cluster s
    // holding strip s; boundary rows cross between clusters through xbuf.
    int strips;
    int pad;
    unsigned char *xbuf;        // per block: 2 sides x 2 step parities x xslot bytes
    unsigned long long xslot;
    ResDone *done;              // completion records (ResJob::done_slot), nullptr: none
    // Job ring and time slices.  Clusters take jobs from the ring in order.  With
    // slice > 0, a cluster whose job has run `slice` more steps while other jobs
    // wait stores the job's state (its rows to the image, its dirty bitmaps to
    // ckbits, its phase to run[]) and puts it back at the ring's tail.
    int *ring;                  // cap entries: job indices
    unsigned *tag;              // per entry: 1 + the round of the ring it was written in
    ResRun *run;                // per job
    uint32_t *ckbits;           // checkpointed dirty bitmaps
    unsigned cap;
    int slice;                  // steps per time slice (a power of two), 0: jobs run to the end once started
};

// A resident launch prepared on the host (device tables uploaded), ready to
// be enqueued any number of times: see resident_prepare / _enqueue /
// _collect / _release.
struct ResidentPrepared {
    int n = 0, C = 0, nw = 0, grid = 0, strips = 0, es = 1;
    size_t smem = 0;
    bool async_alloc = true;
    char *base = nullptr;         // one device allocation holding everything below
    char *live = nullptr, *pristine = nullptr;  // per-run state (stats, control, job ring) and its initial copy
    size_t live_bytes = 0;
    std::vector<int> order;       // launch position -> index in the prepared job list
    ResArgs P;                    // the kernel's argument block
};
// strips > 0: one image (n == 1) over `strips` clusters of C blocks, one
// cooperative launch (the wide mode for images larger than one cluster).
int resident_prepare(const JobSpec *jobs, int n, int C, int nw, const thin_options &opt, cudaStream_t stream,
                     bool async_alloc, ResidentPrepared *R, int strips = 0, ResDone *done = nullptr);
cudaError_t resident_enqueue(const ResidentPrepared &R, cudaStream_t stream);
int resident_collect(const ResidentPrepared &R, const thin_options &opt, cudaStream_t stream, thin_stats *out);
// The public stats of a finished resident job (error: the launch's error word).
void resident_stats(const ResStat &S, int error, const thin_options &opt, thin_stats *o);
void resident_release(ResidentPrepared &R, cudaStream_t stream);
// Smallest cluster of nw-warp blocks whose shared memory holds a w x h image
// of `dtype`, 0 if none.
int resident_cluster_size(int w, int h, int dtype, size_t smem_limit, int nw, int *rows_out, int *rp_out);
// Largest resident cluster on the current device: 16 where it can run, else 8.
int resident_max_cluster(int nw, size_t smem_limit);
// Shared memory one block may take when `blocks` blocks share an SM.
size_t resident_smem_limit(int blocks);
// Wide mode: the fewest strips (clusters of *c_out blocks of nw warps, the
// largest cluster size that works) whose shared memory holds the image, all
// clusters resident at once; 0 if none.
int resident_wide_strips(int w, int h, int dtype, size_t smem_limit, int nw, int *c_out);

// A tiled launch prepared on the host (opaque; thin_tiled.cu).
struct TiledPrepared;
// max_grid > 0 caps the launch at that many blocks (serving keeps the rest of
// the GPU free for the resident launches of its other lanes).
int tiled_prepare(const JobSpec *jobs, int n, const thin_options &opt, cudaStream_t stream, bool async_alloc,
                  TiledPrepared **out, int max_grid = 0);
cudaError_t tiled_enqueue(const TiledPrepared *T, cudaStream_t stream);
int tiled_collect(const TiledPrepared *T, const thin_options &opt, cudaStream_t stream, thin_stats *out);
void tiled_release(TiledPrepared *T, cudaStream_t stream);

// Defaults of the tiled engine for a dtype (tile width/height in pixels, halo).
void tiled_defaults(int dtype, int *tw, int *th, int *halo);

int cuda_status(cudaError_t e);

// Resident launch groups of a batch at most: one per cluster size (1, 2, 4,
// 8, 16) and element size (u8, u16).  Execution::enqueue needs that many helper
// streams, and one event more.
constexpr int kMaxResidentGroups = 10;

// Launch groups of a batch: (cluster size, job indices) for the resident
// engine, job indices for the tiled engine.
struct Grouping {
    int nw = 16;
    std::vector<std::pair<int, std::vector<int>>> resident;
    struct Wide {
        int job, strips, C;
    };
    std::vector<Wide> wide;  // one wide launch each
    std::vector<int> tiled;
};
// allow_wide: large images may take the wide resident mode (a cooperative
// launch over the whole GPU); serving turns it off so that its lanes share
// the GPU.
int group_jobs(const std::vector<JobSpec> &specs, const thin_options &o, Grouping *G, bool allow_wide = true);

// Every launch group of a batch, prepared; enqueue() is device work only
// (resident groups forked onto up to four side streams with events, joined
// back before the tiled group), so it can be captured in a CUDA graph.
struct Execution {
    std::vector<JobSpec> specs;
    thin_options opt;
    bool async = true;
    ResDone *done = nullptr;  // completion records for the resident groups' jobs (JobSpec::done_slot)
    int tiled_max_grid = 0;   // cap on the tiled launch's blocks, 0 = none
    std::vector<ResidentPrepared> res;
    std::vector<std::vector<int>> res_idx;
    std::vector<ResidentPrepared> wide;
    std::vector<int> wide_idx;
    TiledPrepared *tiled = nullptr;
    std::vector<int> tiled_idx;
    int prepare(const std::vector<JobSpec> &specs, const Grouping &G, const thin_options &o, cudaStream_t s,
                bool async_alloc);
    cudaError_t enqueue(cudaStream_t s, cudaStream_t *side, cudaEvent_t *ev) const;
    int collect(cudaStream_t s, thin_stats *out) const;  // out[k] for specs[k]; waits for s
    void release(cudaStream_t s);
};

// Helper streams and events of the calling host thread for Execution::enqueue
// (created once per thread and device, kept until the process exits).
cudaError_t thread_side_streams(cudaStream_t **side, cudaEvent_t **ev);

// Raises a kernel's dynamic shared-memory cap to the device's opt-in maximum.
// Always the same value, so host threads launching the kernel at once with
// different shared-memory sizes never lower the cap under one another.
cudaError_t allow_max_dynamic_smem(const void *kernel);

}  // namespace thin
