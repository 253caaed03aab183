// thin_resident.cu -- the resident lambda-thinning engine: each image lives
// in shared memory for its whole run.
//
// Layout.  Block r of a cluster of C blocks holds image rows [r R, r R + R)
// plus 8 halo rows of each neighbouring block, 16-byte padded.  A block runs 8
// phases on its own (the exact region shrinks by one row per phase into the
// halo), then copies fresh halo rows, and their dirty bits, from its
// neighbours' shared memory (distributed shared memory) between two cluster
// barriers.  A phase writes only points of its own parity and reads only the
// other parities, so the blocks of a cluster never race inside a phase.
// Clusters take images from a device-wide counter, longest first, so images
// of different lengths run side by side without grid-wide synchronisation.
//
// Which points a phase tests.  Per parity there is one bitmap with a bit per
// 4-point group (8 x 2 cell): "a neighbour of one of its points moved since
// the group's last test".  A group that lowers a point sets the bits of the
// groups of the other three parities around it; a phase consumes its own
// parity's bits.  A point none of whose neighbours moved since its last test
// cannot have become lowerable, so the skipped tests change nothing.  Every
// bit is set at the start of a run.  The run stops once three phases in a row
// changed nothing anywhere in the image (its fixed point under the schedule)
// or at the phase cap.
//
// Work in a phase.  Each warp scans its share of the parity's bitmap words
// and appends the groups it finds to one queue of the block; after a block
// barrier the queue is split evenly over ceil(N / 32) warps (at most all 16),
// so a front that crosses only part of the image still keeps the block's
// schedulers busy, and a sparse phase runs on full lanes of a few warps.  A warp whose share is
// larger than 32 groups tests them all first, packing those that lower (with
// their test result) to the front of its share, then lowers them on full
// lanes starting from that result; with fewer it tests and lowers in one
// pass.  One more block barrier ends the phase.
//
// Wide mode.  An image too large for one cluster is spread over all clusters
// of one cooperative launch, a strip each.  Halo rows cross between clusters
// through a global snapshot, and a bounded grid barrier every 8 phases
// carries the stop test.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "thin_common.cuh"
#include "thin_internal.h"
#include "thin_simd.cuh"

namespace cg = cooperative_groups;

namespace thin {

namespace {

// Warps per block: 16, 8 or 4, with 1, 2 or 4 blocks per SM (at most 128
// registers a thread either way).
constexpr int kResMaxWarps = 16;
constexpr int kResStep = 8;  // phases between halo exchanges = halo rows held from each neighbour
// A warp with more queued groups than this tests them all first and lowers
// the ones that qualify on packed lanes; with fewer it lowers as it tests.
// The lowering pass starts from the test pass's result (one byte per group),
// and the common mode (lambda-thinning, F^- = max, (8,4)) has its own build
// of the point test.  Since only neighbours whose test can change are
// marked, most tested groups lower, and re-gathering them in a second pass
// costs more than packing saves: the four-point SIMD path always lowers as it
// tests (the 192-job u8 batch went from 21.8 to 19.8 ms against a threshold
// of 32 groups).  The table path tests first, whatever the count.
constexpr int kTwoPass = 1 << 30;
constexpr bool kOkPass = true;
constexpr bool kFix = true;
// Which neighbours of a lowered point become dirty (marks8 / marks16): 0 all
// eight; 1 those above the point's new value; 2 those also at most its old
// value + lambda (the second bound only outside the wide mode, where it was
// measured to cost more than it saves).  The skipped ones cannot change their
// test result.
#ifndef THIN_RES_MARK
#define THIN_RES_MARK 2
#endif
constexpr int kMark = THIN_RES_MARK;

__device__ const PointTable d_res_point_table = kPointTable;
__device__ const PointTable d_res_point_table48 = kPointTable48;

// Shared-memory map of one block for a job.
constexpr int kOffTabs = 0;      // point tables of (8,4) and (4,8), 2 KiB (the block up to 4 KiB is free)
constexpr int kOffCtrl = 4096;   // control words
constexpr int kOffBar = 4352;    // mbarrier of the row staging
constexpr int kOffRows = 4480;   // image rows (16-byte aligned)
constexpr int kResMaxCluster = 16;  // largest cluster (16 is a non-portable size, used where the device allows)
// Steps (exchanges of halo rows) a job runs before it yields its cluster to a
// waiting job, when a launch has more jobs than clusters: 1024 phases of
// 8-row steps, about 4 ms of a 512^2 job.  A power of two.
constexpr int kResSlice = 128;

struct Ctrl {
    int job;
    long long last;     // last phase in which this block lowered a point, -1 if none
    unsigned long long nlow;
    unsigned long long ntest;
    long long peer_last[kResMaxCluster];  // every block's `last`, pushed by the blocks themselves each phase
    int bar_ok;              // result of the last grid barrier (wide launches)
    unsigned qn[2];          // fill counters of the block's group queue, alternating by scan round
    unsigned fail[2];        // wide launches, cluster leader: a block's grid-barrier wait failed (by step parity)
    int yield;               // cluster leader: the job pauses at this time slice's end
};
static_assert(sizeof(Ctrl) <= kOffBar - kOffCtrl, "control words overlap the mbarrier");

__host__ __device__ inline size_t res_bits_off(int rows, int rp) { return (kOffRows + size_t(rows) * rp + 15) / 16 * 16; }
// four dirty bitmaps (one per parity), then the phase's queue of groups
__host__ __device__ inline size_t res_queue_off(int rows, int rp, int wpr)
{
    return res_bits_off(rows, rp) + size_t(4) * 4 * (rows / 2) * wpr;
}
// A scan round covers min(words, 32 nw) bitmap words of 32 groups each, and
// the block's queue holds every group one round can find: nw x this many
// entries (32 groups per word times min(ceil(words / nw), 32) words).
__host__ __device__ inline int res_warp_queue(int rows, int wpr, int nw)
{
    const int words = (rows / 2) * wpr;
    const int per_warp = (words + nw - 1) / nw;
    return (per_warp < 32 ? per_warp : 32) * 32;
}
__host__ __device__ inline size_t res_smem_bytes(int rows, int rp, int wpr, int nw)
{
    // per warp: 16-bit group codes, then one byte per group (its test result)
    return res_queue_off(rows, rp, wpr) + size_t(3) * nw * res_warp_queue(rows, wpr, nw) + 16;
}

__device__ __forceinline__ unsigned long long res_gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t res_smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ bool res_mbar_wait(uint32_t bar, uint32_t parity, unsigned long long timeout_ns)
{
    const unsigned long long t0 = res_gtimer();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (res_gtimer() - t0 > timeout_ns) return false;
    }
}

// Barrier over all blocks of a wide launch, with a time limit: false if the
// wait ran out (THIN_ERR_TIMEOUT posted) or another block posted an error.
__device__ bool res_grid_barrier(ResCtl *ctl, unsigned nblocks, unsigned long long timeout_ns, int *s_ok)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = &ctl->bar_gen;
        volatile int *err = &ctl->error;
        const unsigned g0 = *gen;
        int ok = 1;
        __threadfence();
        if (atomicAdd(&ctl->bar_count, 1u) == nblocks - 1) {
            atomicExch(&ctl->bar_count, 0u);
            __threadfence();
            atomicAdd(&ctl->bar_gen, 1u);
        } else {
            const unsigned long long t0 = res_gtimer();
            while (*gen == g0) {
                if (*err) {
                    ok = 0;
                    break;
                }
                if (res_gtimer() - t0 > timeout_ns) {
                    atomicCAS(&ctl->error, 0, THIN_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        if (*err) ok = 0;
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// The job ring.  Entry t holds a job once tag[t % cap] == 1 + t / cap.  A pop
// takes the head entry only while head < tail (an empty ring consumes
// nothing, so a cluster that finds it empty may leave); a push appends at the
// tail.  A cluster pushes only a job it paused while others waited, and pops
// again at once, so every pushed job has a taker.  Returns the job, or -1 when
// the ring is empty (or a bounded wait ran out: THIN_ERR_TIMEOUT posted).
__device__ int res_pop(const ResArgs &P)
{
    volatile unsigned *head = &P.ctl->head, *tail = &P.ctl->tail;
    const unsigned long long t0 = res_gtimer();
    for (;;) {
        const unsigned h = *head;
        if (h >= *tail) return -1;
        if (atomicCAS(&P.ctl->head, h, h + 1) != h) {  // another cluster took it: try the next one
            if (res_gtimer() - t0 > P.timeout_ns) {
                atomicCAS(&P.ctl->error, 0, THIN_ERR_TIMEOUT);
                return -1;
            }
            continue;
        }
        const unsigned s = h % P.cap, want = 1u + h / P.cap;
        while (*reinterpret_cast<volatile unsigned *>(&P.tag[s]) != want) {  // its pusher is writing it
            if (res_gtimer() - t0 > P.timeout_ns) {
                atomicCAS(&P.ctl->error, 0, THIN_ERR_TIMEOUT);
                return -1;
            }
        }
        __threadfence();
        return *reinterpret_cast<volatile int *>(&P.ring[s]);
    }
}

__device__ void res_push(const ResArgs &P, int job)
{
    const unsigned t = atomicAdd(&P.ctl->tail, 1u);
    const unsigned s = t % P.cap;
    *reinterpret_cast<volatile int *>(&P.ring[s]) = job;
    __threadfence();
    *reinterpret_cast<volatile unsigned *>(&P.tag[s]) = 1u + t / P.cap;
}

// OR of m into bits[key] (key < 0: nothing to mark).  Combining the lanes
// that name the same word first (__match_any_sync + __reduce_or_sync) was
// measured slower than letting the shared-memory atomics serialise.
__device__ __forceinline__ void or_word(uint32_t *bits, int key, uint32_t m)
{
    if (key >= 0) atomicOr(bits + key, m);
}

// ES: element size of every image of the launch (1: u8, 2: u16).
template <int NW, int ES>
__global__ void __launch_bounds__(NW * 32, kResMaxWarps / NW) k_resident(ResArgs P)
{
    extern __shared__ __align__(128) uint8_t smem[];
    cg::cluster_group cluster = cg::this_cluster();
    const int C = int(cluster.num_blocks());
    const int rank = int(cluster.block_rank());
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t *tabs = reinterpret_cast<uint32_t *>(smem + kOffTabs);
    Ctrl *ctrl = reinterpret_cast<Ctrl *>(smem + kOffCtrl);
    const uint32_t bar = res_smem_u32(smem + kOffBar);
    uint8_t *rows_base = smem + kOffRows;

    for (int i = tid; i < 256; i += blockDim.x) {
        tabs[i] = d_res_point_table.v[i];
        tabs[kTabOffset48 + i] = d_res_point_table48.v[i];
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    uint32_t bar_parity = 0;
    __syncthreads();

    const bool wide = P.strips > 0;
    const int S = wide ? P.strips : 1;                  // strips of the image (clusters)
    const int strip = wide ? int(blockIdx.x) / C : 0;   // this cluster's strip
    const int gb = strip * C + rank;                    // block index within the image
    const int B = S * C;                                // blocks per image
    for (int iter = 0;; ++iter) {
        int job;
        if (wide) {
            if (iter > 0) break;  // a wide launch runs its one image
            job = 0;
        } else {
            if (rank == 0 && tid == 0) ctrl->job = res_pop(P);
            cluster.sync();
            job = cluster.map_shared_rank(ctrl, 0)->job;
            cluster.sync();  // every block has read the leader's word before it may leave or overwrite it
            if (job < 0) break;
        }
        const ResJob J = P.jobs[job];
        constexpr int es = ES;
        const int mode = P.rule | (J.adj << 2);      // F^- reading, operator, adjacency pair
        const bool simd = J.adj == 0;                // (8,4): four points at once (bytes for u8, 16-bit lanes for u16)
        const uint32_t *ptab = tabs + (J.adj ? kTabOffset48 : 0);
        const int R = J.rows, HR = J.hr, RP = J.rp, CW = J.cw, WPR = J.wpr;
        const int LR = R + 2 * HR;   // shared rows: HR halo rows, R own rows, HR halo rows
        const int CRT = LR / 2;      // cell rows held
        const int HC = HR / 2;       // halo cell rows on each side
        const int slot_words = CRT * WPR;
        // dirty[q]: per parity q = 2 (y & 1) + (x & 1), one bit per 4-point group (cell row, column):
        // some neighbour of a point of the group moved since the group's last test
        uint32_t *dirty = reinterpret_cast<uint32_t *>(smem + res_bits_off(LR, RP));
        // the block's queue of the groups found in one scan round (codes, then one test-result byte each)
        const int WQ = res_warp_queue(LR, WPR, NW);
        uint16_t *bqueue = reinterpret_cast<uint16_t *>(smem + res_queue_off(LR, RP, WPR));
        uint8_t *bok = smem + res_queue_off(LR, RP, WPR) + size_t(2) * NW * WQ;
        const int row0 = gb * R;         // first own image row
        const int ybase = row0 - HR;     // image row of shared row 0
        const int rowb = J.w * es;
        const char *gimg = reinterpret_cast<const char *>(J.img);

        // ---- stage own and halo rows that exist in the image (with slices on, they may have been
        // written by the cluster that paused the job: order them before this block's bulk copies)
        if (P.slice > 0) asm volatile("fence.proxy.async.global;" ::: "memory");
        const int ya = max(0, ybase), yb = min(J.h, ybase + LR);
        const int nload = max(0, yb - ya);
        if (J.bulk && nload > 0) {
            if (tid == 0)
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                             "r"(uint32_t(nload * rowb))
                             : "memory");
            __syncthreads();
            for (int r = tid; r < nload; r += blockDim.x) {
                const uint32_t dst = res_smem_u32(rows_base + size_t(ya - ybase + r) * RP + 16);
                const char *src = gimg + size_t(ya + r) * J.pitch;
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                    "l"(src), "r"(uint32_t(rowb)), "r"(bar)
                    : "memory");
            }
            if (!res_mbar_wait(bar, bar_parity, P.timeout_ns)) {
                if (tid == 0) atomicCAS(&P.ctl->error, 0, THIN_ERR_TIMEOUT);
                res_mbar_wait(bar, bar_parity, P.timeout_ns);  // let copies in flight land (bounded)
            }
            bar_parity ^= 1u;
        } else {
            for (int e = tid; e < nload * rowb; e += blockDim.x) {
                const int r = e / rowb, c = e - r * rowb;
                rows_base[size_t(ya - ybase + r) * RP + 16 + c] = uint8_t(__ldcg(gimg + size_t(ya + r) * J.pitch + c));
            }
        }
        // a fresh job tests every group in the first phase of its parity; a resumed one restores the
        // dirty bitmaps of its checkpoint (written by another SM: read through L2)
        ResRun run;
        run.resumed = 0;
        if (P.slice > 0) {
            const volatile ResRun &vr = P.run[job];
            run.g = vr.g;
            run.last = vr.last;
            run.resumed = vr.resumed;
        }
        if (run.resumed) {
            const uint32_t *ck = P.ckbits + J.ck + size_t(rank) * 4 * slot_words;
            for (int i = tid; i < 4 * slot_words; i += blockDim.x) dirty[i] = __ldcg(ck + i);
        } else {
            for (int i = tid; i < 4 * slot_words; i += blockDim.x) dirty[i] = 0xffffffffu;
        }
        const long long last0 = run.resumed ? run.last : -1;
        if (tid == 0) {
            ctrl->last = last0;
            ctrl->nlow = 0;
            ctrl->ntest = 0;
            ctrl->qn[0] = 0u;
            ctrl->qn[1] = 0u;
            ctrl->fail[0] = 0u;
            ctrl->fail[1] = 0u;
        }
        if (tid < kResMaxCluster) ctrl->peer_last[tid] = last0;
        // No block may push its last change into a peer (end of the first step) before that peer has
        // set its array above: the arrays must agree, or the blocks could take different stop
        // decisions and their cluster barriers stop pairing.
        cluster.sync();

        const uint32_t Mwpr = WPR > 1 ? 0xffffffffu / uint32_t(WPR) + 1u : 0u;
        const uint32_t Mcw = CW > 1 ? 0xffffffffu / uint32_t(CW) + 1u : 0u;

        long long g = run.resumed ? run.g : P.start_phase;
        unsigned qround = 0;  // scan rounds so far: selects the queue counter
        unsigned steps = 0;   // steps of this job on this cluster
        int converged = 0;
        bool paused = false;
        int nlow = 0, ntest = 0;
        for (;;) {  // steps of H phases between exchanges of halo rows
            const long long done = g - P.start_phase;
            if (P.max_phases >= 0 && done >= P.max_phases) break;
            const int Hs = (P.max_phases >= 0 && P.max_phases - done < J.steph) ? int(P.max_phases - done) : J.steph;
            for (int j = 0; j < Hs; ++j, ++g) {
                const int p = int(g & 3), px = p & 1, py = p >> 1;
                uint32_t *dp = dirty + p * slot_words;
                // rows whose points are exact in this phase: own rows and Hs-1-j halo rows
                const int rr = B > 1 ? Hs - 1 - j : 0;
                const int ylo = max(1, row0 - rr), yhi = min(J.h - 2, row0 + R - 1 + rr);
                // the groups of the other three parities holding a neighbour to test again become
                // dirty.  A: byte k holds the ring directions (bit 0 E, 1 NE, 2 N, 3 NW, 4 W, 5 SW,
                // 6 S, 7 SE) of point k's neighbours to mark; 0: nothing to mark.  E and W neighbours
                // are in the row's other column parity, N and S in the other row parity, the
                // diagonals in the fourth.  For px == 0 the W side of point 0 is in the cell to the
                // left; for px == 1 the E side of point 3 is in the cell to the right.
                const int qrow = 2 * py + (px ^ 1), qcol = 2 * (py ^ 1) + px, qdiag = 2 * (py ^ 1) + (px ^ 1);
                auto mark = [&](int cr, int cc, uint32_t A) {
                    const uint32_t rs = A & (px ? 0x10111111u : 0x11111101u);  // same cell: E, W
                    const uint32_t as = A & (px ? 0x080a0a0au : 0x0a0a0a02u);  // NE, NW
                    const uint32_t bs = A & (px ? 0x20a0a0a0u : 0xa0a0a080u);  // SE, SW
                    const uint32_t rx = A & (px ? 0x01000000u : 0x00000010u);  // the cell beside
                    const uint32_t ax = A & (px ? 0x02000000u : 0x00000008u);
                    const uint32_t bx = A & (px ? 0x80000000u : 0x00000020u);
                    const int w = cc >> 5, b = cc & 31;
                    const uint32_t mc = 1u << b;
                    const bool edge = px ? b == 31 : b == 0;  // the cell beside is in the next word
                    const uint32_t mx = edge ? 0u : (px ? mc << 1 : mc >> 1);
                    const uint32_t mrow = (rs ? mc : 0u) | (rx ? mx : 0u);
                    const uint32_t ma = (as ? mc : 0u) | (ax ? mx : 0u);
                    const uint32_t mb = (bs ? mc : 0u) | (bx ? mx : 0u);
                    const int ca = cr - 1 + py, cb = cr + py;  // cell rows of rows y - 1, y + 1
                    const bool va = ca >= 0, vb = cb < CRT;
                    or_word(dirty, mrow ? qrow * slot_words + cr * WPR + w : -1, mrow);
                    or_word(dirty, va && (A & 0x04040404u) ? qcol * slot_words + ca * WPR + w : -1, mc);
                    or_word(dirty, va && ma ? qdiag * slot_words + ca * WPR + w : -1, ma);
                    or_word(dirty, vb && (A & 0x40404040u) ? qcol * slot_words + cb * WPR + w : -1, mc);
                    or_word(dirty, vb && mb ? qdiag * slot_words + cb * WPR + w : -1, mb);
                    if (edge && (rx | ax | bx)) {  // the group across a word boundary (rare)
                        const int ws = px ? w + 1 : w - 1;
                        const uint32_t ms = px ? 1u : 0x80000000u;
                        if (rx) atomicOr(&dirty[qrow * slot_words + cr * WPR + ws], ms);
                        if (va && ax) atomicOr(&dirty[qdiag * slot_words + ca * WPR + ws], ms);
                        if (vb && bx) atomicOr(&dirty[qdiag * slot_words + cb * WPR + ws], ms);
                    }
                };
                auto where = [&](int code, int &cr, int &cc, uint32_t &vm, uint32_t &in) {
                    cr = CW > 1 ? int(__umulhi(uint32_t(code), Mcw)) : code;
                    cc = code - cr * CW;
                    const int y = ybase + 2 * cr + py;
                    vm = 0;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const int x = 8 * cc + px + 2 * kk;
                        vm |= (x >= 1 && x <= J.w - 2 ? 1u : 0u) << (8 * kk);
                    }
                    in = (y >= row0 && y < row0 + R) ? vm : 0u;  // own points count
                };
                bool moved_own = false;
                // the (8,4) point test on four points at once, in the common mode's own build where it applies
                auto test_item = [&](const uint8_t *rb, int pxx, uint32_t vm) -> uint32_t {
                    if constexpr (ES == 1) {
                        return (kFix && mode == 0) ? test_u8<0>(rb - RP, rb, rb + RP, pxx, vm, J.lam, mode)
                                                   : test_u8(rb - RP, rb, rb + RP, pxx, vm, J.lam, mode);
                    } else {
                        const uint16_t *r16 = reinterpret_cast<const uint16_t *>(rb);
                        const int rp16 = RP / 2;
                        return (kFix && mode == 0) ? test_u16<0>(r16 - rp16, r16, r16 + rp16, pxx, vm, J.lam, mode)
                                                   : test_u16(r16 - rp16, r16, r16 + rp16, pxx, vm, J.lam, mode);
                    }
                };
                // the lowering loop on four points (ok: a first test's result, or ~0u to test first);
                // aff receives the neighbours to mark
                auto lower_item = [&](uint8_t *rb, int pxx, uint32_t vm, uint32_t in, uint32_t ok, uint32_t &aff) -> uint32_t {
                    if constexpr (ES == 1) {
                        if (ok == ~0u)
                            return (kFix && mode == 0)
                                       ? item_u8<0, kMark>(rb - RP, rb, rb + RP, pxx, vm, in, J.lam, mode, nlow, aff, !wide)
                                       : item_u8<-1, kMark>(rb - RP, rb, rb + RP, pxx, vm, in, J.lam, mode, nlow, aff, !wide);
                        return (kFix && mode == 0)
                                   ? item_u8_tested<0, kMark>(rb - RP, rb, rb + RP, pxx, vm, in, ok, J.lam, mode, nlow, aff, !wide)
                                   : item_u8_tested<-1, kMark>(rb - RP, rb, rb + RP, pxx, vm, in, ok, J.lam, mode, nlow, aff, !wide);
                    } else {
                        uint16_t *r16 = reinterpret_cast<uint16_t *>(rb);
                        const int rp16 = RP / 2;
                        return (kFix && mode == 0)
                                   ? item_u16<0, kMark>(r16 - rp16, r16, r16 + rp16, pxx, vm, in, ok, J.lam, mode, nlow, aff, !wide)
                                   : item_u16<-1, kMark>(r16 - rp16, r16, r16 + rp16, pxx, vm, in, ok, J.lam, mode, nlow, aff, !wide);
                    }
                };
                // A scan round: warp w takes the round's bitmap words 32 w .. 32 w + 31 of this parity
                // (one per lane; a small bitmap keeps only the first warps scanning), consumes their bits
                // and appends the groups it found to the block's queue.  After a block barrier the queue
                // is split over the warps, and each warp tests and lowers its share on its own: no other
                // block barrier until the end of the phase (or of the round, when the bitmap needs several).
                for (int r0 = 0; r0 < slot_words; r0 += 32 * NW) {
                    {
                        const int wi = r0 + warp * 32 + lane;  // 32 consecutive words a warp: few warps scan
                        uint32_t d = 0;
                        int cr = 0;
                        if (wi < slot_words) {
                            cr = WPR > 1 ? int(__umulhi(uint32_t(wi), Mwpr)) : wi;
                            const int i = wi - cr * WPR;
                            const int y = ybase + 2 * cr + py;
                            if (y >= ylo && y <= yhi) {
                                const int valid = CW - 32 * i;
                                d = dp[wi] & (valid >= 32 ? 0xffffffffu : ((1u << valid) - 1u));
                            }
                            if (dp[wi]) dp[wi] = 0u;
                        }
                        const int cnt = __popc(d);
                        int incl = cnt;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const int v = __shfl_up_sync(0xffffffffu, incl, o);
                            if (lane >= o) incl += v;
                        }
                        const int wsum = __shfl_sync(0xffffffffu, incl, 31);
                        if (wsum) {
                            int base = 0;
                            if (lane == 31) base = int(atomicAdd(&ctrl->qn[qround & 1], unsigned(wsum)));
                            int pos = __shfl_sync(0xffffffffu, base, 31) + incl - cnt;
                            const int cbase = (wi - cr * WPR) * 32 + cr * CW;
                            while (d) {
                                const int bb = __ffs(d) - 1;
                                d &= d - 1;
                                bqueue[pos++] = uint16_t(cbase + bb);
                            }
                        }
                    }
                    __syncthreads();
                    const int N = int(*reinterpret_cast<volatile unsigned *>(&ctrl->qn[qround & 1]));
                    if (tid == 0) ctrl->qn[(qround + 1) & 1] = 0u;  // last read in the previous round
                    ++qround;
                    // The shares go to as few warps as give every warp a full chunk of 32 (all 16 when
                    // there are more than 512 groups): a sparse phase then issues its groups on full
                    // lanes from about one warp per scheduler instead of a few lanes of every warp.
                    const int act = min(NW, (N + 31) >> 5);
                    const int qa = warp < act ? (N * warp) / act : N;
                    const int nq = warp < act ? (N * (warp + 1)) / act - qa : 0;  // queue slots qa .. qa + nq - 1
                    uint16_t *wqueue = bqueue + qa;
                    uint8_t *wok = bok + qa;
                    if (nq > 0) {
                        int nl = nq;
                        if (!simd || nq > kTwoPass) {
                            // test first; the groups that lower are packed to the front of the share
                            // (in place: a chunk's slots are read before any of them is written)
                            nl = 0;
                            for (int kb = 0; kb < nq; kb += 32) {
                                const int k = kb + lane;
                                bool lowers = false;
                                int code = 0, gcr = 0, gcc = 0;
                                uint32_t tmoved = 0;
                                if (k < nq) {
                                    code = wqueue[k];
                                    uint32_t vm, in;
                                    where(code, gcr, gcc, vm, in);
                                    ntest += __popc(in);
                                    uint8_t *rb = rows_base + size_t(2 * gcr + py) * RP + 16 + size_t(8 * es) * gcc;
                                    if (simd) {
                                        const uint32_t okb = test_item(rb, px, vm);
                                        lowers = okb != 0;
                                        code |= int((okb | (okb >> 7) | (okb >> 14) | (okb >> 21)) & 0xfu) << 16;
                                    } else {
                                        if constexpr (ES == 2)
                                            tmoved = item_table<uint16_t>(reinterpret_cast<const uint16_t *>(rb - RP),
                                                                          reinterpret_cast<uint16_t *>(rb),
                                                                          reinterpret_cast<const uint16_t *>(rb + RP), px,
                                                                          vm, in, ptab, J.lam, mode, nlow);
                                        else
                                            tmoved = item_table<uint8_t>(rb - RP, rb, rb + RP, px, vm, in, ptab, J.lam,
                                                                         mode, nlow);
                                        if (tmoved & in) moved_own = true;
                                    }
                                }
                                if (!simd) mark(gcr, gcc, tmoved * 0xffu);  // the table path marks every neighbour
                                const unsigned bal = __ballot_sync(0xffffffffu, lowers);
                                if (lowers) {
                                    const int at = nl + __popc(bal & ((1u << lane) - 1u));
                                    wqueue[at] = uint16_t(code);
                                    wok[at] = uint8_t(code >> 16);  // which of the four points passed the test
                                }
                                nl += __popc(bal);
                            }
                            __syncwarp();
                            if (!simd) nl = 0;
                        }
                        // lower them (u8, (8,4)); with few groups the loop's first test is the only one
                        for (int kb = 0; kb < nl; kb += 32) {
                            const int k = kb + lane;
                            int gcr = 0, gcc = 0;
                            uint32_t moved = 0, aff = 0;
                            if (k < nl) {
                                const int code = wqueue[k];
                                uint32_t vm, in;
                                where(code, gcr, gcc, vm, in);
                                if (nq <= kTwoPass) ntest += __popc(in);
                                uint8_t *rb = rows_base + size_t(2 * gcr + py) * RP + 16 + size_t(8 * es) * gcc;
                                if (kOkPass && nq > kTwoPass) {  // tested in the first pass: start lowering at once
                                    const uint32_t o4 = wok[k];
                                    const uint32_t okb = (o4 & 1u) | ((o4 & 2u) << 7) | ((o4 & 4u) << 14) | ((o4 & 8u) << 21);
                                    moved = lower_item(rb, px, vm, in, okb, aff);
                                } else {
                                    moved = lower_item(rb, px, vm, in, ~0u, aff);
                                }
                                if (moved & in) moved_own = true;
                            }
                            mark(gcr, gcc, aff);
                        }
                        __syncwarp();
                    }
                    if (r0 + 32 * NW < slot_words) __syncthreads();  // the next round refills the queue
                }
                if (__syncthreads_or(moved_own) && tid == 0) ctrl->last = g;
            }
            // ---- end of a step: every block's last change, then the stop test
            __syncthreads();
            const int sp = int(steps & 1);  // buffer of this step in the exchange snapshot
            ++steps;
            long long lc = -1;
            if (wide) {
                // boundary rows (and their dirty bits) for the neighbouring strips go to a global
                // snapshot; a grid barrier; then every block reads the global last change
                const int vrow = RP / 16;
                const int dwords = 4 * (HC + 1) * WPR;
                auto publish = [&](int side, int row_from, int cell_from) {
                    unsigned char *slot = P.xbuf + ((size_t(gb) * 2 + side) * 2 + sp) * P.xslot;
                    uint4 *dst = reinterpret_cast<uint4 *>(slot);
                    const uint4 *src = reinterpret_cast<const uint4 *>(rows_base + size_t(row_from) * RP);
                    for (int e = tid; e < HR * vrow; e += blockDim.x) __stcg(dst + e, src[e]);
                    uint32_t *dd = reinterpret_cast<uint32_t *>(slot + size_t(HR) * RP);
                    for (int e = tid; e < dwords; e += blockDim.x) {
                        const int q = e / ((HC + 1) * WPR), o = e - q * (HC + 1) * WPR;
                        __stcg(dd + e, dirty[q * slot_words + cell_from * WPR + o]);
                    }
                };
                if (rank == 0 && strip > 0) publish(0, HR, HC - 1);              // my first own rows, for the strip above
                if (rank == C - 1 && strip + 1 < S) publish(1, R, R / 2);        // my last own rows, for the strip below
                if (tid == 0) atomicMax(&P.ctl->gl_last, ctrl->last);
                __threadfence();
                const bool bar_ok = res_grid_barrier(P.ctl, gridDim.x, P.timeout_ns, &ctrl->bar_ok);
                // The blocks of a cluster leave the step loop together or not at all, so that their
                // cluster barriers keep pairing up: a block whose wait failed posts it to the leader.
                Ctrl *lead = cluster.map_shared_rank(ctrl, 0);
                if (tid == 0 && !bar_ok) atomicOr(&lead->fail[sp], 1u);
                cluster.sync();
                const bool cluster_ok = *reinterpret_cast<volatile unsigned *>(&lead->fail[sp]) == 0u;
                if (rank == 0 && tid == 0) ctrl->fail[sp ^ 1] = 0u;  // read by the cluster one step ago
                if (!cluster_ok) break;
                lc = *reinterpret_cast<volatile long long *>(&P.ctl->gl_last);
            } else {
                if (tid < C) cluster.map_shared_rank(ctrl, tid)->peer_last[rank] = ctrl->last;  // push to every block
                cluster.sync();
                for (int q = 0; q < C; ++q) lc = max(lc, ctrl->peer_last[q]);
            }
            if (g - P.start_phase >= 4 && lc < g - 3) {  // three quiet phases everywhere: fixed point
                converged = 1;
                break;
            }
            if (P.max_phases >= 0 && g - P.start_phase >= P.max_phases) break;
            if (B > 1) {
                // halo rows and their dirty bits from the blocks above and below (their own rows);
                // the marks a neighbour made on my first or last row (from its own rows, which I
                // do not follow to the end of a step) are merged into mine
                const int vrow = RP / 16;
                if (gb > 0) {
                    const uint4 *src;
                    const uint32_t *nd;
                    int nd_from;  // first cell row to read in nd
                    if (rank > 0) {
                        src = reinterpret_cast<const uint4 *>(cluster.map_shared_rank(rows_base, rank - 1) + size_t(R) * RP);
                        nd = cluster.map_shared_rank(dirty, rank - 1);
                        nd_from = R / 2;
                    } else {  // the strip above published its last rows
                        const unsigned char *slot = P.xbuf + ((size_t(gb - 1) * 2 + 1) * 2 + sp) * P.xslot;
                        src = reinterpret_cast<const uint4 *>(slot);
                        nd = reinterpret_cast<const uint32_t *>(slot + size_t(HR) * RP);
                        nd_from = -1;
                    }
                    uint4 *dst = reinterpret_cast<uint4 *>(rows_base);
                    for (int e = tid; e < HR * vrow; e += blockDim.x) dst[e] = nd_from >= 0 ? src[e] : __ldcg(src + e);
                    for (int e = tid; e < 4 * (HC + 1) * WPR; e += blockDim.x) {
                        // neighbour cell rows R/2 .. R/2 + HC -> mine 0 .. HC
                        const int q = e / ((HC + 1) * WPR), o = e - q * (HC + 1) * WPR;
                        const uint32_t v = nd_from >= 0 ? nd[q * slot_words + nd_from * WPR + o] : __ldcg(nd + e);
                        uint32_t &d = dirty[q * slot_words + o];
                        d = o < (HC - 1) * WPR ? v : (d | v);  // the two cell rows at the seam: both blocks' marks
                    }
                }
                if (gb + 1 < B) {
                    const uint4 *src;
                    const uint32_t *nd;
                    int nd_from;
                    if (rank + 1 < C) {
                        src = reinterpret_cast<const uint4 *>(cluster.map_shared_rank(rows_base, rank + 1) + size_t(HR) * RP);
                        nd = cluster.map_shared_rank(dirty, rank + 1);
                        nd_from = HC - 1;
                    } else {  // the strip below published its first rows
                        const unsigned char *slot = P.xbuf + ((size_t(gb + 1) * 2 + 0) * 2 + sp) * P.xslot;
                        src = reinterpret_cast<const uint4 *>(slot);
                        nd = reinterpret_cast<const uint32_t *>(slot + size_t(HR) * RP);
                        nd_from = -1;
                    }
                    uint4 *dst = reinterpret_cast<uint4 *>(rows_base + size_t(HR + R) * RP);
                    for (int e = tid; e < HR * vrow; e += blockDim.x) dst[e] = nd_from >= 0 ? src[e] : __ldcg(src + e);
                    for (int e = tid; e < 4 * (HC + 1) * WPR; e += blockDim.x) {
                        // neighbour cell rows HC - 1 .. 2 HC - 1 -> mine HC + R/2 - 1 .. 2 HC + R/2 - 1
                        const int q = e / ((HC + 1) * WPR), o = e - q * (HC + 1) * WPR;
                        const uint32_t v = nd_from >= 0 ? nd[q * slot_words + nd_from * WPR + o] : __ldcg(nd + e);
                        uint32_t &d = dirty[q * slot_words + (HC + R / 2 - 1) * WPR + o];
                        d = o >= 2 * WPR ? v : (d | v);
                    }
                }
                if (C > 1) cluster.sync();  // nobody changes its own rows before its neighbours have copied them
                else __syncthreads();
            }
            // end of a time slice: pause the job if other jobs wait for a cluster (the leader decides for
            // the whole cluster; its word is next written a slice later, after many cluster barriers)
            if (P.slice > 0 && (steps & unsigned(P.slice - 1)) == 0u) {
                if (rank == 0 && tid == 0)
                    ctrl->yield = *reinterpret_cast<volatile unsigned *>(&P.ctl->head) <
                                  *reinterpret_cast<volatile unsigned *>(&P.ctl->tail);
                cluster.sync();
                if (cluster.map_shared_rank(ctrl, 0)->yield) {
                    paused = true;
                    break;
                }
            }
        }
        // ---- results
        nlow = __reduce_add_sync(0xffffffffu, nlow);
        ntest = __reduce_add_sync(0xffffffffu, ntest);
        if (lane == 0 && nlow) atomicAdd(&ctrl->nlow, (unsigned long long)nlow);
        if (lane == 0 && ntest) atomicAdd(&ctrl->ntest, (unsigned long long)ntest);
        __syncthreads();
        // the job's fields used from here on are read again (fewer registers live through the steps)
        const ResJob &Jg = P.jobs[job];
        {
            const int ra = max(row0, 1), rb = min(row0 + R, J.h - 1);  // border rows never change
            char *gout = reinterpret_cast<char *>(Jg.img);
            const unsigned long long pitch = Jg.pitch;
            if (Jg.bulk) {
                const int vpr = rowb / 16;
                for (int e = tid; e < max(0, rb - ra) * vpr; e += blockDim.x) {
                    const int r = e / vpr, c = e - r * vpr;
                    *reinterpret_cast<uint4 *>(gout + size_t(ra + r) * pitch + 16 * c) =
                        *reinterpret_cast<const uint4 *>(rows_base + size_t(ra + r - ybase) * RP + 16 + 16 * c);
                }
            } else {
                for (int e = tid; e < max(0, rb - ra) * rowb; e += blockDim.x) {
                    const int r = e / rowb, c = e - r * rowb;
                    gout[size_t(ra + r) * pitch + c] = char(rows_base[size_t(ra + r - ybase) * RP + 16 + c]);
                }
            }
        }
        if (paused) {
            // checkpoint: the rows went to the image above; the dirty bitmaps, the counts and the
            // phase to resume at go to global memory, then the job goes back to the ring's tail
            uint32_t *ckw = P.ckbits + Jg.ck + size_t(rank) * 4 * slot_words;
            for (int i = tid; i < 4 * slot_words; i += blockDim.x) __stcg(ckw + i, dirty[i]);
            if (tid == 0) {
                ResStat &St = P.st[job];
                atomicAdd(&St.lowered, ctrl->nlow);
                atomicAdd(&St.tested, ctrl->ntest);
                if (rank == 0) {
                    long long lc = -1;
                    for (int q = 0; q < C; ++q) lc = max(lc, ctrl->peer_last[q]);
                    volatile ResRun &vr = P.run[job];
                    vr.g = g;
                    vr.last = lc;
                    vr.resumed = 1;
                }
            }
            __threadfence();
            asm volatile("fence.proxy.async.global;" ::: "memory");       // the rows are read back by bulk copies
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes before the next bulk copy
            cluster.sync();  // every block's rows and bitmaps are out
            if (rank == 0 && tid == 0) res_push(P, job);
            continue;
        }
        if (tid == 0) {
            ResStat &St = P.st[job];
            atomicAdd(&St.lowered, ctrl->nlow);
            atomicAdd(&St.tested, ctrl->ntest);
            if (gb == 0) {
                long long lc = -1;
                if (wide) lc = *reinterpret_cast<volatile long long *>(&P.ctl->gl_last);
                else
                    for (int q = 0; q < C; ++q) lc = max(lc, ctrl->peer_last[q]);
                St.last_change = lc;
                St.phases = g - P.start_phase;
                St.converged = converged;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes before the next bulk copy
        const int done_slot = Jg.done_slot;
        const bool post = P.done != nullptr && done_slot >= 0;
        if (post) __threadfence_system();  // this block's rows are out before the leader posts the record
        cluster.sync();  // nobody reads this job's rows or control words any more
        if (post && rank == 0 && tid == 0) {
            // completion record: the job's stats (every block added its counts before the cluster barrier),
            // then the flag, released at system scope for the host that polls it
            const volatile ResStat &S = P.st[job];
            ResDone *d = P.done + done_slot;
            d->st.lowered = S.lowered;
            d->st.tested = S.tested;
            d->st.last_change = S.last_change;
            d->st.phases = S.phases;
            d->st.converged = S.converged;
            d->st.error = 0;
            d->error = *reinterpret_cast<volatile int *>(&P.ctl->error);
            __threadfence_system();
            asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(&d->flag), "r"(1u) : "memory");
        }
    }
}

// Launch shape of k_resident<NW, ES>: as many clusters of C blocks as fit at
// once (each loops over the job queue), at most one per job.
template <int NW, int ES>
cudaError_t resident_shape(int C, int n, size_t smem, int *grid)
{
    cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void *>(k_resident<NW, ES>));
    if (e == cudaSuccess && C > 8)
        e = cudaFuncSetAttribute(reinterpret_cast<const void *>(k_resident<NW, ES>),
                                 cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof cfg);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(NW * 32);
    cfg.dynamicSmemBytes = smem;
    cfg.gridDim = dim3(C);
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveClusters(&clusters, k_resident<NW, ES>, &cfg);
    if (e == cudaSuccess && clusters < 1) e = cudaErrorInvalidConfiguration;
    *grid = C * std::min(clusters, n);
    return e;
}

// Wide launches are cooperative: the clusters of one image wait on one
// another at every step, so all of them must be resident at once.
template <int NW, int ES>
cudaError_t resident_launch(int C, int grid, size_t smem, cudaStream_t stream, const ResArgs &P)
{
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof cfg);
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeCooperative;
    attr[1].val.cooperative = 1;
    cfg.blockDim = dim3(NW * 32);
    cfg.gridDim = dim3(grid);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = P.strips > 0 ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, k_resident<NW, ES>, P);
}

// The launch shape for blocks of nw warps (16: the one shape the engine uses) and element size es.
cudaError_t resident_shape_for(int nw, int es, int C, int n, size_t smem, int *grid)
{
    if (nw != kResMaxWarps) return cudaErrorInvalidValue;
    return es == 2 ? resident_shape<kResMaxWarps, 2>(C, n, smem, grid) : resident_shape<kResMaxWarps, 1>(C, n, smem, grid);
}

}  // namespace

// Largest cluster the device can run with blocks of nw warps and smem_limit
// bytes of shared memory each: 16 where clusters of 16 (a non-portable size)
// can be resident, else 8.  Asked once per device.
int resident_max_cluster(int nw, size_t smem_limit)
{
    static int cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 8;
    }
    if (!cached[dev]) {
        int g1 = 0, g2 = 0;
        const cudaError_t e1 = resident_shape_for(nw, 1, kResMaxCluster, 1, smem_limit, &g1);
        const cudaError_t e2 = resident_shape_for(nw, 2, kResMaxCluster, 1, smem_limit, &g2);
        cudaGetLastError();
        cached[dev] = (e1 == cudaSuccess && e2 == cudaSuccess && g1 == kResMaxCluster && g2 == kResMaxCluster)
                          ? kResMaxCluster
                          : 8;
    }
    return cached[dev];
}

// Smallest cluster (1, 2, 4, 8, or 16 where the device allows it, blocks of
// nw warps) whose shared memory holds the image; 0 if none.
int resident_cluster_size(int w, int h, int dtype, size_t smem_limit, int nw, int *rows_out, int *rp_out)
{
    const int es = dtype == THIN_U16 ? 2 : 1;
    const int rp = int((size_t(w) * es + 15) / 16 * 16) + 32;
    const int cw = (w + 7) / 8, wpr = (cw + 31) / 32;
    const int cmax = resident_max_cluster(nw, smem_limit);
    for (int C = 1; C <= cmax; C *= 2) {
        int rows = (h + C - 1) / C;
        rows += rows & 1;
        const int held = rows + (C > 1 ? 2 * std::min(kResStep, rows) : 0);  // halo: see resident_run
        if (held / 2 * cw > 65535) continue;  // queue codes are 16-bit
        if (res_smem_bytes(held, rp, wpr, nw) <= smem_limit) {
            if (rows_out) *rows_out = rows;
            if (rp_out) *rp_out = rp;
            return C;
        }
    }
    return 0;
}

// Wide mode: the largest cluster size C (8, 4, 2, 1) and the fewest strips
// S (clusters) whose shared memory holds the image with all S clusters
// resident at once (clusters must fit within a GPC, so large clusters cannot
// use every SM).  Returns S and stores C, or 0 if none.
int resident_wide_strips(int w, int h, int dtype, size_t smem_limit, int nw, int *c_out)
{
    const int es = dtype == THIN_U16 ? 2 : 1;
    const int rp = int((size_t(w) * es + 15) / 16 * 16) + 32;
    const int cw = (w + 7) / 8, wpr = (cw + 31) / 32;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int max_blocks = sms * (kResMaxWarps / nw);
    for (int C = 8; C >= 1; C /= 2) {
        for (int S = 2; S * C <= max_blocks; ++S) {
            int rows = (h + S * C - 1) / (S * C);
            rows += rows & 1;
            const int held = rows + 2 * std::min(kResStep, rows);
            if (held / 2 * cw > 65535) continue;  // queue codes are 16-bit
            const size_t smem = res_smem_bytes(held, rp, wpr, nw);
            if (smem > smem_limit) continue;
            // every cluster of the launch must be resident at once
            int grid = 0;
            const cudaError_t e = resident_shape_for(nw, es, C, S, smem, &grid);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return 0;
            }
            if (grid == S * C) {
                if (c_out) *c_out = C;
                return S;
            }
            break;  // more strips of this size fit even less: try smaller clusters
        }
    }
    return 0;
}

// Shared memory a block may take when `blocks` blocks share an SM.
size_t resident_smem_limit(int blocks)
{
    int dev = 0, optin = 0, per_sm = 0, reserved = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    size_t lim = size_t(optin > 0 ? optin : 48 * 1024);
    if (blocks > 1 && per_sm > 0) lim = std::min(lim, size_t(per_sm) / blocks - size_t(reserved));
    return lim;
}

// Host-side preparation of one launch: job table (longest first), stats and
// control words, and their pristine copies, all in one device allocation.
int resident_prepare(const JobSpec *jobs, int n, int C, int nw, const thin_options &opt, cudaStream_t stream,
                     bool async_alloc, ResidentPrepared *R, int strips, ResDone *done)
{
    *R = ResidentPrepared();
    R->n = n;
    R->C = C;
    R->nw = nw;
    R->strips = strips;
    R->async_alloc = async_alloc;
    if (strips > 0 && n != 1) return THIN_ERR_ARG;  // a wide launch runs one image
    const int B = strips > 0 ? strips * C : C;      // blocks per image
    if (nw != kResMaxWarps || n < 1) return THIN_ERR_ARG;
    R->es = elem_size(jobs[0].dtype);
    for (int k = 1; k < n; ++k)
        if (elem_size(jobs[k].dtype) != R->es) return THIN_ERR_ARG;  // one element size per launch
    const size_t limit = resident_smem_limit(kResMaxWarps / nw);
    std::vector<ResJob> rj(n);
    size_t smem = 0;
    for (int k = 0; k < n; ++k) {
        const JobSpec &J = jobs[k];
        ResJob &r = rj[k];
        std::memset(&r, 0, sizeof r);
        const int es = elem_size(J.dtype);
        r.img = reinterpret_cast<unsigned long long>(J.img);
        r.pitch = J.pitch;
        r.w = J.w;
        r.h = J.h;
        r.dtype = J.dtype;
        r.lam = J.lam;
        int rows = (J.h + B - 1) / B;
        rows += rows & 1;
        r.rows = rows;
        // halo rows must be own rows of the neighbouring block: never deeper than a block's share
        r.steph = std::min(kResStep, rows);
        r.hr = B > 1 ? r.steph : 0;
        r.rp = int((size_t(J.w) * es + 15) / 16 * 16) + 32;
        r.cw = (J.w + 7) / 8;
        r.wpr = (r.cw + 31) / 32;
        r.bulk = (reinterpret_cast<uintptr_t>(J.img) % 16 == 0) && (J.pitch % 16 == 0) && ((size_t(J.w) * es) % 16 == 0);
        r.index = k;
        r.adj = J.adj;
        r.done_slot = strips > 0 ? -1 : J.done_slot;
        const int held = r.rows + 2 * r.hr;
        const size_t need = res_smem_bytes(held, r.rp, r.wpr, nw);
        if (need > limit || held / 2 * r.cw > 65535) return THIN_ERR_ARG;
        smem = std::max(smem, need);
    }
    // longest-first: larger lambda and larger images tend to run longer
    std::vector<int> order(n);
    for (int k = 0; k < n; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const double ca = double(rj[a].w) * rj[a].h * (1.0 + rj[a].lam), cb = double(rj[b].w) * rj[b].h * (1.0 + rj[b].lam);
        return ca > cb;
    });
    std::vector<ResJob> sorted(n);
    for (int k = 0; k < n; ++k) sorted[k] = rj[order[k]];
    R->order = order;
    R->smem = smem;

    // launch shape first: time slices only pay when more jobs than clusters wait
    const int want = strips > 0 ? strips : n;  // clusters wanted
    cudaError_t e = resident_shape_for(nw, R->es, C, want, smem, &R->grid);
    if (e != cudaSuccess) return cuda_status(e);
    if (strips > 0 && R->grid < B) return THIN_ERR_ARG;  // not all strips fit at once
    const int clusters = std::max(1, R->grid / C);
    const int slice = (strips == 0 && n > clusters) ? kResSlice : 0;
    const unsigned cap = unsigned(n + clusters);  // ring entries: queued jobs plus one pop in flight per cluster
    size_t ck_words = 0;
    if (slice > 0)
        for (auto &r : sorted) {
            r.ck = ck_words;
            ck_words += size_t(C) * 4 * ((r.rows + 2 * r.hr) / 2) * r.wpr;
        }

    // one allocation: job table | live state (stats, control, per-job run, ring tags, ring) | its
    // pristine copy, the same layout | checkpoints | wide-mode exchange slots
    auto up = [](size_t v) { return (v + 255) / 256 * 256; };
    const size_t o_jobs = 0;
    const size_t l_st = 0, l_ctl = up(sizeof(ResStat) * n), l_run = l_ctl + up(sizeof(ResCtl));
    const size_t l_tag = l_run + up(sizeof(ResRun) * n), l_ring = l_tag + up(sizeof(unsigned) * cap);
    const size_t live_bytes = l_ring + up(sizeof(int) * cap);
    const size_t o_live = up(sizeof(ResJob) * n);
    const size_t o_prist = o_live + live_bytes;
    const size_t o_ck = o_prist + live_bytes;
    // wide: per block, 2 sides x 2 step parities of (halo rows + their dirty words)
    size_t xslot = 0;
    if (strips > 0) {
        const ResJob &r = rj[0];
        xslot = up(size_t(r.hr) * r.rp + size_t(4) * (r.hr / 2 + 1) * r.wpr * 4);
    }
    const size_t o_x = o_ck + up(ck_words * 4);
    const size_t total = o_x + xslot * 4 * size_t(B);
    e = async_alloc ? cudaMallocAsync(reinterpret_cast<void **>(&R->base), total, stream)
                    : cudaMalloc(reinterpret_cast<void **>(&R->base), total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        R->base = nullptr;
        return THIN_ERR_OOM;
    }
    // the pristine live state: fresh stats, every job queued in order
    std::vector<char> prist(live_bytes, 0);
    ResStat *st0 = reinterpret_cast<ResStat *>(prist.data() + l_st);
    for (int k = 0; k < n; ++k) st0[k].last_change = -1;
    ResCtl *ctl0 = reinterpret_cast<ResCtl *>(prist.data() + l_ctl);
    ctl0->gl_last = -1;
    ctl0->head = 0;
    ctl0->tail = unsigned(n);
    ResRun *run0 = reinterpret_cast<ResRun *>(prist.data() + l_run);
    for (int k = 0; k < n; ++k) run0[k].last = -1;
    unsigned *tag0 = reinterpret_cast<unsigned *>(prist.data() + l_tag);
    int *ring0 = reinterpret_cast<int *>(prist.data() + l_ring);
    for (int k = 0; k < n; ++k) {
        ring0[k] = k;
        tag0[k] = 1u;  // written in round 0
    }
    e = cudaMemcpyAsync(R->base + o_jobs, sorted.data(), sizeof(ResJob) * n, cudaMemcpyHostToDevice, stream);
    // (pageable sources: each copy has taken its bytes when it returns)
    if (e == cudaSuccess) e = cudaMemcpyAsync(R->base + o_prist, prist.data(), live_bytes, cudaMemcpyHostToDevice, stream);
    R->live = R->base + o_live;
    R->pristine = R->base + o_prist;
    R->live_bytes = live_bytes;

    ResArgs &P = R->P;
    std::memset(&P, 0, sizeof P);
    P.jobs = reinterpret_cast<const ResJob *>(R->base + o_jobs);
    P.st = reinterpret_cast<ResStat *>(R->live + l_st);
    P.ctl = reinterpret_cast<ResCtl *>(R->live + l_ctl);
    P.run = reinterpret_cast<ResRun *>(R->live + l_run);
    P.tag = reinterpret_cast<unsigned *>(R->live + l_tag);
    P.ring = reinterpret_cast<int *>(R->live + l_ring);
    P.ckbits = slice > 0 ? reinterpret_cast<uint32_t *>(R->base + o_ck) : nullptr;
    P.cap = cap;
    P.slice = slice;
    P.njobs = n;
    P.rule = test_mode(opt);  // F^- reading and operator
    P.start_phase = opt.start_phase;
    P.max_phases = opt.max_phases;
    P.timeout_ns = 2000000000ull;
    P.strips = strips;
    P.xbuf = strips > 0 ? reinterpret_cast<unsigned char *>(R->base + o_x) : nullptr;
    P.xslot = xslot;
    P.done = strips > 0 ? nullptr : done;
    if (const char *t = std::getenv("THIN_TIMEOUT_NS")) P.timeout_ns = std::strtoull(t, nullptr, 10);
    return e == cudaSuccess ? THIN_OK : cuda_status(e);
}

// Resets the stats and control words from their pristine copies and
// launches: device work only, so it can be captured in a CUDA graph.
cudaError_t resident_enqueue(const ResidentPrepared &R, cudaStream_t stream)
{
    const cudaError_t e = cudaMemcpyAsync(R.live, R.pristine, R.live_bytes, cudaMemcpyDeviceToDevice, stream);
    if (e != cudaSuccess) return e;
    return R.es == 2 ? resident_launch<kResMaxWarps, 2>(R.C, R.grid, R.smem, stream, R.P)
                     : resident_launch<kResMaxWarps, 1>(R.C, R.grid, R.smem, stream, R.P);
}

// Waits for the stream and writes the stats of job k (the caller's order) to out[k].
int resident_collect(const ResidentPrepared &R, const thin_options &opt, cudaStream_t stream, thin_stats *out)
{
    const int n = R.n;
    std::vector<ResStat> st(n);
    ResCtl ctl;
    cudaError_t e = cudaMemcpyAsync(st.data(), R.P.st, sizeof(ResStat) * n, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ctl, R.P.ctl, sizeof ctl, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_status(e);
    int rc = THIN_OK;
    for (int k = 0; k < n; ++k) {
        thin_stats &o = out[R.order[k]];
        resident_stats(st[k], ctl.error, opt, &o);
        if (o.status != THIN_OK && rc == THIN_OK) rc = o.status;
    }
    return rc;
}

void resident_stats(const ResStat &S, int error, const thin_options &opt, thin_stats *o)
{
    std::memset(o, 0, sizeof *o);
    o->converged = S.converged && !error;
    o->status = error ? error : (o->converged ? THIN_OK : THIN_ERR_NOT_CONVERGED);
    o->phases = S.phases;
    o->lowered = (int64_t)S.lowered;
    o->last_change_phase = S.last_change;
    o->end_phase = opt.start_phase + S.phases;
    o->tiles_visited = 0;
    o->steps = S.phases;
    o->tested = (int64_t)S.tested;
}

void resident_release(ResidentPrepared &R, cudaStream_t stream)
{
    if (R.base) {
        if (R.async_alloc) cudaFreeAsync(R.base, stream);
        else cudaFree(R.base);
    }
    R.base = nullptr;
}

}  // namespace thin
