/*
 * thin.h -- C-ABI of the GB300 grayscale lambda-thinning library (libthin.so).
 *
 * The operation: grayscale lambda-thinning under (8,4)- or (4,8)-adjacency
 * (Sec. 2.1: n for the sections of F, nbar for their complements).  Every
 * lambda-destructible point (Sec. 2.1: a destructible point, or a
 * k-divergent point with at least k-1 lower components c such that
 * F(x) - F^-(c) <= lambda) is lowered to alpha^-(x, F), the largest value among
 * its strictly lower 8-neighbours (Sec. 2.1), repeatedly until no such point
 * remains (the lowering loop of Sec. 2.2, with lambda-destructible points in
 * place of lambda-deletable, non-lambda-end ones).  The paper's own
 * lambda-skeleton is selected with thin_options.op.
 *
 * The order of lowering is fixed so that the result is unique: a 2x2-parity
 * subfield schedule.  Phase g (a global phase index, 0, 1, 2, ...) visits the
 * interior points with 2*(y & 1) + (x & 1) == g mod 4; such points are
 * pairwise not 8-adjacent, so a phase equals any sequential order over its
 * points.  Within its phase a point is lowered until it is no longer
 * lambda-destructible.  The run stops at the schedule's fixed point: three
 * phases in a row that change nothing mean every point has been tested since
 * its neighbours last moved.  The engines check this every few phases, so
 * stats.phases may run a few phases past stats.last_change_phase + 3.  Border
 * pixels (x = 0, x = w-1, y = 0, y = h-1) are read as neighbours and never
 * written.
 *
 * Layout: an image is h rows of w pixels, row-major, rows `pitch_bytes` apart;
 * pixel (x, y) is column x of row y.  u8 images hold uint8_t, u16 images
 * uint16_t (the full 0..65535 range is allowed).
 *
 * Ownership: image memory belongs to the caller, who keeps it alive until the
 * work queued on `stream` has finished.  Calls are asynchronous on `stream`
 * (a cudaStream_t passed as void*; NULL = the legacy default stream) unless a
 * stats pointer is given: then the call waits for the stream and fills the
 * stats before returning.  Scratch memory is taken from, and returned to,
 * the CUDA stream-ordered allocator on the same stream.
 *
 * Errors: every entry point returns THIN_OK (0) or a negative THIN_ERR_* code
 * and leaves the image untouched when it rejects its arguments.  Errors found
 * on the device (a bounded wait that ran out) are reported in stats.status.
 */
#ifndef THIN_H
#define THIN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define THIN_OK 0
#define THIN_ERR_ARG (-1)           /* bad pointer, size, pitch, dtype, lambda or option */
#define THIN_ERR_UNSUPPORTED (-2)   /* an option the library was compiled without */
#define THIN_ERR_OOM (-3)           /* scratch allocation failed */
#define THIN_ERR_NOT_CONVERGED (-4) /* stopped by max_phases before stability */
#define THIN_ERR_TIMEOUT (-5)       /* a bounded device wait ran out */
#define THIN_ERR_CUDA (-6)          /* a CUDA runtime call failed */
#define THIN_EAGAIN (-7)            /* serving: the admission queue or the pinned staging is full; retry */
#define THIN_ERR_TOO_LARGE (-8)     /* thin_run_noalloc: the image needs more than its fixed scratch;
                                       serving: the image alone exceeds the budget or the staging */

typedef enum { THIN_U8 = 0, THIN_U16 = 1 } thin_dtype;
/* Adjacency pair (n, nbar) of Sec. 2.1: (8,4) or (4,8).  Under (4,8), T+
 * counts 4-components of Gamma^+ that hold a 4-neighbour of x, T-- counts
 * 8-components of Gamma^--, and an end point has one 4-neighbour in F_k. */
typedef enum { THIN_ADJ_8_4 = 0, THIN_ADJ_4_8 = 1 } thin_adj;

/* Reading of F^-(c) in the lambda rule (Sec. 2.1 leaves F^- undefined):
 * THIN_RULE_MAX takes the largest value of F over the component c (default),
 * THIN_RULE_MIN the smallest.  THIN_RULE_MIN is an unpinned reading: the
 * paper fixes no example that tells the two apart (they agree on components
 * of one value), so its results are checked against the oracle's same
 * reading only. */
typedef enum { THIN_RULE_MAX = 0, THIN_RULE_MIN = 1 } thin_rule;

/* The operator (Sec. 2.1-2.2), both lowering points to alpha^-(x, F) in the
 * same subfield schedule:
 * THIN_OP_THINNING  lambda-thinning: lower lambda-destructible points (default);
 * THIN_OP_SKELETON  lambda-skeleton, the paper's operator: lower points that
 *                   are lambda-deletable (lambda-destructible, or a peak point,
 *                   T+ = 0, with F(x) - alpha^- <= lambda) and not lambda-end
 *                   (an end point of F_k, k = F(x), with F(x) - alpha^- > lambda). */
typedef enum { THIN_OP_THINNING = 0, THIN_OP_SKELETON = 1 } thin_op;

/* Kernel family.  RESIDENT holds each image in shared memory for its whole
 * run: in one thread-block cluster of up to 16 blocks (images up to about
 * 2.4 MB: 1550 x 1550 u8, 1100 x 1100 u16; 1.25 MB where the device runs
 * clusters of 8 at most), or, in the wide mode, in several clusters of one
 * cooperative launch (one block per SM, clusters of 8, 4, 2 or 1 blocks,
 * whichever lets every strip be resident) that exchange boundary rows every
 * 8 phases: images up to about 30 MB.  TILED streams 64 x 32 tiles through
 * shared memory (any size).  AUTO picks RESIDENT for images that fit a
 * cluster, the wide mode for up to two larger images in a call, and TILED
 * for the rest.  NAIVE runs one launch per phase straight from global memory
 * (the reference slice). */
typedef enum {
    THIN_KERNEL_AUTO = 0,
    THIN_KERNEL_NAIVE = 1,
    THIN_KERNEL_TILED = 2,
    THIN_KERNEL_RESIDENT = 3
} thin_kernel;

typedef struct {
    int32_t rule;        /* thin_rule */
    int32_t kernel;      /* thin_kernel */
    int32_t tile_w;      /* tiled engine: tile width in pixels, 0 = default (64); multiple of 16, 16..224 */
    int32_t tile_h;      /* tiled engine: tile height, 0 = default (32); even, >= 8, tile_h + 2 halo <= 256 */
    int32_t halo;        /* tiled engine: phases per tile visit = halo width, 0 = default (8); 3..8 when a u16
                            image is in the call, else 3..16; below min(tile_w, tile_h).  A shape that does not
                            fit one block's shared memory returns THIN_ERR_ARG */
    int32_t reserved;    /* 0.  Test hook: 1 makes block 0 of the tiled engine skip its first grid barrier, so
                            that the bounded wait runs out and the call reports THIN_ERR_TIMEOUT */
    int64_t start_phase; /* global phase index of the first phase (resume), >= 0 */
    int64_t max_phases;  /* stop after this many phases; < 0 = run to stability */
    int32_t op;          /* thin_op */
    int32_t reserved2;   /* 0 */
} thin_options;

typedef struct {
    int32_t status;            /* THIN_OK, THIN_ERR_NOT_CONVERGED or THIN_ERR_TIMEOUT */
    int32_t converged;         /* 1 if a quiet stretch of four phases was seen */
    int64_t phases;            /* phases run by this call */
    int64_t lowered;           /* lowering steps F(x) := alpha^- performed */
    int64_t last_change_phase; /* global index of the last phase that lowered a point; -1 if none */
    int64_t end_phase;         /* global phase index to resume from */
    int64_t tiles_visited;     /* tile visits of the tiled kernel (0 for NAIVE) */
    int64_t steps;             /* tile steps (tiled) or rounds of four phases (naive) */
    int64_t tested;            /* point tests made: a point is tested in a phase of its parity only
                                  if a neighbour moved since its last test (all points in the first
                                  four phases); the work behind the sweep rate */
} thin_stats;

/* Fills *opt with the defaults (rule MAX, AUTO kernel, default tiles, phase 0, no cap, lambda-thinning). */
void thin_default_options(thin_options *opt);

/*
 * Lambda-thin one image in place (Sec. 2.1-2.2).
 *   img_dev      device pointer to pixel (0, 0); u8 images need no alignment,
 *                u16 images 2-byte alignment
 *   w, h         width and height in pixels; w <= 0 or h <= 0 with w, h >= 0
 *                is an empty image (no-op); images narrower or lower than 3
 *                pixels have no interior point and are left unchanged
 *   pitch_bytes  distance between rows, >= w * element size
 *   dt           THIN_U8 or THIN_U16
 *   lambda       the contrast parameter, an integer >= 0 (Sec. 2.1)
 *   adj          THIN_ADJ_8_4 or THIN_ADJ_4_8
 *   stream       cudaStream_t as void*
 *   opt          options, NULL = defaults
 *   out          stats, NULL = fully asynchronous call
 */
int thin_run(void *img_dev, int w, int h, size_t pitch_bytes, thin_dtype dt, uint32_t lambda,
             thin_adj adj, void *stream, const thin_options *opt, thin_stats *out);

/* One image of a batch. */
typedef struct {
    void *img_dev;      /* device pointer, caller-owned, thinned in place */
    int32_t w, h;       /* width, height in pixels */
    size_t pitch;       /* row pitch in bytes */
    int32_t dtype;      /* thin_dtype */
    uint32_t lambda;    /* per-image lambda */
} thin_job;

/*
 * Lambda-thin n independent images of any sizes, dtypes and lambdas in one
 * call.  Images that fit one thread-block cluster's shared memory run on the
 * resident engine, one launch per cluster size, the launches side by side
 * on streams forked from `stream` and joined back into it.  Images too large
 * for a cluster run in the wide resident mode, one launch each, when there
 * are at most two of them (any number with THIN_KERNEL_RESIDENT); otherwise
 * they go to one persistent launch of the tiled engine, after the resident
 * launches.  Every such launch loops on the device until its images are
 * stable.  THIN_KERNEL_TILED sends every image to the tiled engine;
 * THIN_KERNEL_NAIVE thins the images one after another, as thin_run does
 * with that kernel.  Each image gets exactly the result thin_run
 * gives it alone.  opt applies to every image (its start_phase too).  out:
 * array of n stats or NULL.  n == 0 is a no-op.
 */
int thin_batch(const thin_job *jobs, int n, thin_adj adj, void *stream, const thin_options *opt,
               thin_stats *out);

/* ----------------------------------------------------------------------
 * Batch plans: thin_batch prepared once and run many times as one CUDA graph
 * (the graph-captured form of the batch drive; the paper has no counterpart,
 * its drive is the CPU FIFO of Sec. 3.2).
 *
 * thin_plan_create does all host work of a thin_batch call once (checks,
 * launch groups, device job tables, tensor maps) and captures the device
 * work of one run into a CUDA graph: per-run resets, the resident engine's
 * launch groups side by side, the tiled engine after them.  Images that go
 * to the tiled engine get a tile shape and halo depth chosen by
 * thin_autotune on the largest of them, unless opt sets tile_w, tile_h or
 * halo.
 * thin_plan_launch enqueues that graph: every image is thinned in place, with
 * exactly the result thin_batch gives.  The images must stay at the same
 * device addresses while the plan exists; relaunching thins whatever the
 * images hold then (restore them first to repeat a run).  Launches of one
 * plan must not overlap on the device (they share the plan's tables).
 * -------------------------------------------------------------------- */
typedef struct thin_plan thin_plan;

/* jobs, n, adj, opt as for thin_batch (the NAIVE kernel returns
 * THIN_ERR_UNSUPPORTED).  The plan owns device memory (stream-ordered allocator) until it
 * is destroyed.  Synchronous: returns once the plan is ready. */
int thin_plan_create(const thin_job *jobs, int n, thin_adj adj, const thin_options *opt, thin_plan **out);

/* Enqueues one run on stream (asynchronous). */
int thin_plan_launch(thin_plan *p, void *stream);

/* Waits for stream and writes the stats of the plan's last run, one per job
 * (n entries).  Returns THIN_OK or the first non-OK status, as thin_batch. */
int thin_plan_stats(thin_plan *p, void *stream, thin_stats *out);

/* The tiled engine's tile shape and halo depth the plan chose by autotuning
 * (all 0 when it has no tiled images or the caller fixed them). */
int thin_plan_tiling(const thin_plan *p, int *tile_w, int *tile_h, int *halo);

/* Waits for the plan's last launch to finish (not for other work on the
 * device), then frees the plan. */
int thin_plan_destroy(thin_plan *p);

/*
 * Autotuner of the tiled engine (temporal blocking, Sec. 2.2's lowering loop
 * run h phases per tile visit; the paper has no counterpart).  Times every
 * candidate tile shape and halo depth h (phases per visit) on a scratch copy
 * of the image -- the image itself is not changed -- and writes the fastest
 * into opt->tile_w, opt->tile_h and opt->halo.  The other fields of *opt are
 * kept and used for the trials (rule, op, start_phase); the trials run under
 * (8,4) adjacency, whichever pair the image is later thinned with.
 * trial_phases bounds each trial (< 0: every trial runs to stability).
 * best_ms (may be NULL) receives the winner's time.  Synchronous.
 * Candidates: 64x32 (h 8, 6, 4), 128x32, 64x64, 128x64, 32x32, 96x48,
 * 128x16, 224x32, 48x64 (h 8), 64x16 (h 6).  THIN_ERR_ARG for an image
 * without interior points.
 */
int thin_autotune(const void *img_dev, int w, int h, size_t pitch_bytes, thin_dtype dt, uint32_t lambda,
                  void *stream, int64_t trial_phases, thin_options *opt, float *best_ms);

/*
 * The 256-entry point-test table the kernels use, written to out[256]
 * (host memory, no GPU needed).  Entry m describes a point whose strictly
 * lower neighbours form the ring mask m (bit i = neighbour i in the order E,
 * NE, N, NW, W, SW, S, SE):
 *   bits 0-2   T+  = number of 8-components of the other neighbours (Sec. 2.1)
 *   bits 3-5   T-- = number of 4-components of the lower neighbours holding a
 *              4-neighbour of x (Sec. 2.1, complement side of (8,4))
 *   bits 6-29  3-bit field per neighbour i at bit 6+3i: 1 + the index of its
 *              counted T-- component, 0 if none
 *   bit 30     destructible (T+ == 1 and T-- == 1)
 *   bit 31     k-divergent (T-- >= 2)
 */
void thin_point_table(uint32_t out[256]);

/* The same table for either adjacency pair; thin_point_table is
 * thin_point_table_adj(THIN_ADJ_8_4, out). */
void thin_point_table_adj(thin_adj adj, uint32_t out[256]);

/*
 * thin_run_noalloc: thin_run with the tiled engine for callers that cannot
 * allocate device memory when they call in: an application that hands all
 * device memory to its own allocator at start-up (a further cudaMalloc would
 * fail or eat into that budget), or a loop with a fixed time budget that may
 * not call into the allocator, which can have to map new memory or wait for
 * the device.  The paper has no counterpart: this is a property of the
 * library, not of the method.
 *
 * Arguments, layout, result and stats are those of thin_run (the kernel
 * option is ignored: the tiled engine always runs).  Scratch memory comes
 * from one array of THIN_NOALLOC_SCRATCH_BYTES that the library declares in
 * device memory; every GPU that loads the library holds it until the process
 * exits.  The call allocates nothing.
 *   - An image whose scratch (a second image-sized buffer, one more if its
 *     rows are not 16-byte aligned, 4 bytes per 8 x 2 pixels of change stamps
 *     and a few words per 64 x 32 tile) does not fit returns
 *     THIN_ERR_TOO_LARGE and is left untouched.  16 MiB holds, for example,
 *     a 3500 x 3500 u8 or a 2500 x 2500 u16 image with 16-byte aligned rows
 *     (unaligned rows need the extra buffer: 2048 x 2048 u8 still fits).
 *   - The first call on a device looks up the array's device address (again
 *     after the device's context is created anew, e.g. after cudaDeviceReset);
 *     make that first call before any stream capture begins.
 *   - Every call uses the same array and overwrites what the previous call
 *     left there (the call itself resets everything it reads).  Calls that
 *     can overlap on the GPU -- on different streams, or from several host
 *     threads -- race on the array and give wrong results: serialise them.
 */
#define THIN_NOALLOC_SCRATCH_BYTES (16u << 20)
int thin_run_noalloc(void *img_dev, int w, int h, size_t pitch_bytes, thin_dtype dt, uint32_t lambda,
                     thin_adj adj, void *stream, const thin_options *opt, thin_stats *out);

/* Library version string. */
const char *thin_version(void);

/* ----------------------------------------------------------------------
 * Serving: continuous batching under a device-memory budget (the batch and
 * serve drive of the GPU form; the paper's own drive is the FIFO of Sec. 3.2,
 * run by CPU threads).
 *
 * A server owns eight worker lanes (host threads, each with its own CUDA
 * streams) on the device that is current at thin_serve_create.  submit copies
 * the host image into a pinned host buffer and returns at once with a ticket.
 * Requests wait in two queues: images that fit one thread-block cluster's
 * shared memory (the resident engine), and larger ones (the tiled engine).
 * An idle lane admits requests of one queue in arrival order while the slot
 * count and the byte budget allow, at most max_slots / 8 of them (a request
 * that does not fit waits at the head of its queue); at most two lanes at a
 * time take from the large queue, and each of their tiled launches uses at
 * most a quarter of the SMs, so small requests keep running beside them.
 * The lane allocates the device images, copies them in and launches them as
 * one batch (never the wide mode, so that the lanes share the GPU).  Each
 * resident image is retired as soon as it is finished -- its result copied
 * back and its bytes and slot returned -- while the rest of its batch still
 * runs; tiled images retire when their batch ends.  Queued requests are
 * admitted by the next idle lane as slots and memory free up, and run on the
 * device beside the batches already there.  Host staging is one pinned arena
 * allocated at create (a quarter of the device budget, clamped to
 * 256 MiB .. 4 GiB), so submit makes no CUDA allocation.  Each image gets
 * exactly the result thin_run gives it alone (rule MAX, default options,
 * (8,4)-adjacency).  The server's functions may be called from any host
 * threads.
 * -------------------------------------------------------------------- */
typedef struct thin_server thin_server;

/* device_budget_bytes: cap on the device bytes charged by admitted requests;
 * a request is charged twice its image (16-byte aligned rows) plus 1/4 byte
 * a pixel plus 64 KiB, which covers the engines' scratch.  max_slots: cap on
 * requests admitted at once.  queue_cap: cap on requests waiting for
 * admission.  Returns THIN_ERR_ARG for a zero budget or cap, THIN_ERR_CUDA
 * if no device is usable, THIN_ERR_OOM if the pinned staging arena cannot be
 * allocated. */
int thin_serve_create(size_t device_budget_bytes, int max_slots, int queue_cap, thin_server **out);

/* Queue one host image (any host memory: it is copied before the call
 * returns; rows pitch bytes apart).  *ticket identifies it.  Returns
 * THIN_EAGAIN when queue_cap requests are already waiting or the pinned
 * staging arena is full (nothing queued; try again later),
 * THIN_ERR_TOO_LARGE when the image alone is charged more than the budget or
 * is larger than the staging arena.
 * Images narrower or lower than 3 pixels finish at once, unchanged. */
int thin_serve_submit(thin_server *s, const void *host_img, int w, int h, size_t pitch,
                      thin_dtype dt, uint32_t lambda, uint64_t *ticket);

/* Non-blocking: *done = 0 while the request is queued or running.  Once it
 * has finished, *done = 1, the result is copied to host_out (rows out_pitch
 * bytes apart), stats (may be NULL) are filled and the ticket is retired; the
 * return value is then the request's status (THIN_OK, or the error its batch
 * met).  An unknown or retired ticket returns THIN_ERR_ARG. */
int thin_serve_poll(thin_server *s, uint64_t ticket, void *host_out, size_t out_pitch, int *done,
                    thin_stats *stats);

/* Blocks up to timeout_ms for a finished request that has not been polled
 * yet and stores its ticket (finished requests come out in the order they
 * finished).  Returns THIN_EAGAIN on timeout.  The server remembers the last
 * 4 x (max_slots + queue_cap) finishes only. */
int thin_serve_wait_any(thin_server *s, int timeout_ms, uint64_t *ticket);

/* Stops the lanes (each finishes the batch it admitted; requests still
 * waiting for admission are dropped) and frees everything, tickets included. */
int thin_serve_destroy(thin_server *s);

#ifdef __cplusplus
}
#endif

#endif /* THIN_H */
