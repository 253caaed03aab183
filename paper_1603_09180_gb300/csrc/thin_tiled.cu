// thin_tiled.cu -- the tiled lambda-thinning engine.
//
// One persistent cooperative launch runs the whole subfield schedule for any
// number of images.  The schedule advances in steps of H phases (temporal
// blocking).  In a step every active tile of every image is visited by one
// warp: a TMA 2-D tile load stages the tile with a halo of H pixels in the
// warp's shared memory, the warp advances H consecutive phases there (the exact
// region shrinks by one pixel ring per phase, so the TW x TH interior is exact
// after H phases) and stores the interior to the other buffer of a ping-pong
// pair.  A grid barrier separates steps.
//
// Which points a phase must test.  A point whose 8 neighbours did not change
// since its own last test (four phases earlier) cannot have become
// lambda-destructible, so skipping it changes nothing.  Changes are recorded
// per cell of 8 x 2 pixels as the global index of the last phase that lowered
// a point in the cell; these stamps persist per image between tile visits.  A
// group of four points is tested at phase g only if a cell of its 3 x 3 cell
// neighbourhood changed at a phase >= g - 3.  Stamps start at the first phase
// of the run, so every point is tested during the first four phases.
//
// Which tiles a step visits.  At the start of a step (phase g0) every unstable
// point lies next to a point that changed during phases g0-3 .. g0-1, and
// unstable points spread by at most one pixel per phase, so a tile none of
// whose 3x3 block of tiles changed in those three phases cannot change during
// the next H <= min(TW, TH) - 1 phases: it is skipped.  A tile that changed at
// all in a step is also visited in the next one, which keeps both ping-pong
// buffers equal on every skipped tile.  The first step (and any step starting
// within three phases of the first) visits every tile.  When a step visits no
// tile the image is at its fixed point and both buffers hold it.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "thin_common.cuh"
#include "thin_internal.h"
#include "thin_simd.cuh"

namespace thin {

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = 32 * kWarps;
constexpr int kMinHalo = 3;
constexpr int kNever = -(1 << 30);  // stamp of a cell that never changes

struct ImgDesc {
    CUtensorMap map[2];          // TMA descriptors of buffer 0 and buffer 1
    unsigned long long buf[2];   // device pointers of the ping-pong pair
    unsigned long long pitch;    // row pitch of both buffers, bytes
    unsigned long long user;     // caller's image
    unsigned long long user_pitch;
    unsigned long long cells;    // int32 stamps, cells_x x cells_y, relative to the first phase
    int w, h, dtype;
    unsigned lam;
    int tiles_x, tiles_y, tile_base, copy_in;
    int cells_x, cells_y, adj, pad1;
};

struct ImgStat {
    unsigned long long lowered;
    unsigned long long tiles_visited;
    unsigned long long tested;  // point tests on tile interiors
    long long last_change;  // global phase index, -1 if none
    int last_step;          // last step that visited a tile of this image
    int last_listed;        // last step for which a tile of this image was listed
};

struct Ctl {
    unsigned bar_count;
    unsigned bar_gen;
    int error;
    int steps;
    unsigned list_count[3];
    unsigned next_item[3];  // per step (mod 3): items claimed beyond the first one of every warp
};

// Shared memory of one warp: tile buffer, cell stamps (with a border ring of
// never-changing cells), work queue and mbarrier.
struct WarpLayout {
    int tile_bytes;   // TMA box bytes + 16 (word reads past the last row stay inside)
    int cell_off;     // offset of the stamps
    int queue_off;    // offset of the queue (u16 entries)
    int bar_off;      // offset of the mbarrier
    int bytes;        // total, 128-aligned
    int ccols, crows; // stamp grid including the border ring
};

struct EngineArgs {
    const ImgDesc *imgs;
    ImgStat *st;
    int *listed;       // per tile: last step index it was appended for
    unsigned *lists;   // 3 lists of total_tiles entries each
    Ctl *ctl;
    int n_imgs;
    int total_tiles;
    int tw, th, halo, hr, rule;  // hr: halo rows in shared memory (halo rounded up to even)
    long long start_phase;
    long long max_phases;
    unsigned long long timeout_ns;
    WarpLayout wl;
    int debug;         // 1: block 0 never arrives at the first barrier (timeout test)
};

__device__ const PointTable d_point_table = kPointTable;
__device__ const PointTable d_point_table48 = kPointTable48;

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of an mbarrier; false after timeout_ns.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long timeout_ns)
{
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = gtimer();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (gtimer() - t0 > timeout_ns) return false;
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar,
                                            uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Grid barrier with a time limit.  Returns false if the wait ran out or an
// error was posted; then ctl->error is set.
__device__ bool grid_barrier(Ctl *ctl, unsigned nblocks, unsigned long long timeout_ns, bool skip_arrive,
                             int *s_flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = &ctl->bar_gen;
        volatile int *err = &ctl->error;
        const unsigned g = *gen;
        int ok = 1;
        __threadfence();
        asm volatile("fence.proxy.async.global;" ::: "memory");
        bool last = false;
        if (!skip_arrive) last = atomicAdd(&ctl->bar_count, 1u) == nblocks - 1;
        if (last) {
            atomicExch(&ctl->bar_count, 0u);
            __threadfence();
            atomicAdd(&ctl->bar_gen, 1u);
        } else {
            const unsigned long long t0 = gtimer();
            while (*gen == g) {
                if (*err) {
                    ok = 0;
                    break;
                }
                if (gtimer() - t0 > timeout_ns) {
                    atomicCAS(&ctl->error, 0, THIN_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        asm volatile("fence.proxy.async.global;" ::: "memory");
        if (*err) ok = 0;
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

__device__ __forceinline__ int find_image(const ImgDesc *imgs, int n, int gt)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (imgs[mid].tile_base <= gt)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Exact n / d for n, d < 2^16 with M = floor(2^32 / d) + 1 (M unused when d == 1).
__device__ __forceinline__ int div_small(int n, int d, uint32_t M)
{
    return d == 1 ? n : int(__umulhi(uint32_t(n), M));
}

__device__ __forceinline__ uint32_t div_magic(int d)
{
    return d > 1 ? 0xffffffffu / uint32_t(d) + 1u : 0u;
}

// Per-visit constants, held in registers.
struct Visit {
    int w, h;           // image size
    uint32_t lam;
    int rule;
    int x0, y0;         // tile origin in the image
    int tw, th;         // tile size
    int H, Hs, hr;      // halo, phases to run, halo rows in shared memory
    int pad;            // elements of left pad in shared memory (16 B)
    long long g0;       // global index of the first phase of the step
    long long start;    // global index of the first phase of the run
};

// Hs phases of the subfield schedule on a staged tile, visited by one warp.
// Shared cell (sx, sy) holds image pixel (x0 - pad + sx, y0 - hr + sy); stamp
// cell (cx, cy) of the grid covers shared columns 8 (cx - 1) .. + 7 and rows
// 2 (cy - 1) .. + 1 (one border ring of never-changing cells).  Phase j updates
// the points of its parity within distance Hs-1-j of the tile and off the
// image border; after Hs phases the tile interior is exact.
template <typename T>
__device__ void visit_phases(T *tile, int bw, int32_t *cells, int ccols, uint16_t *queue, const Visit &V,
                             const uint32_t *tabs, int &nlow, int &chg_j, int &ntest)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt_lanes = (1u << lane) - 1u;
    for (int j = 0; j < V.Hs; ++j) {
        const long long g = V.g0 + j;
        const int rel = int(g - V.start);
        const int p = int(g & 3);
        const int px = p & 1, py = p >> 1;
        const int r = V.Hs - 1 - j;
        const int lox = max(V.x0 - r, 1), hix = min(V.x0 + V.tw + r - 1, V.w - 2);
        const int loy = max(V.y0 - r, 1), hiy = min(V.y0 + V.th + r - 1, V.h - 2);
        const int ya = loy + ((py - loy) & 1);
        const int nrows = hiy >= ya ? (hiy - ya) / 2 + 1 : 0;
        const int slo = lox - V.x0 + V.pad, shi = hix - V.x0 + V.pad;
        const int qlo = slo >> 3;
        const int nq = shi >= slo ? (shi >> 3) - qlo + 1 : 0;
        const uint32_t Mq = div_magic(nq);
        const int sra = ya - V.y0 + V.hr;
        const int items = nrows * nq;
        // 1. the items whose 3x3 stamp cells changed in the last three phases
        int qn = 0;
        for (int base = 0; base < items; base += 32) {
            const int it = base + lane;
            bool dirty = false;
            int code = 0;
            if (it < items) {
                const int rk = div_small(it, nq, Mq);
                const int q = qlo + it - rk * nq;
                const int sr = sra + 2 * rk;
                const int32_t *cp = cells + ((sr >> 1) + 1) * ccols + q + 1;
                int m = max(max(cp[-ccols - 1], cp[-ccols]), cp[-ccols + 1]);
                m = max(m, max(max(cp[-1], cp[0]), cp[1]));
                m = max(m, max(max(cp[ccols - 1], cp[ccols]), cp[ccols + 1]));
                dirty = m >= rel - 3;
                code = (sr << 6) | q;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, dirty);
            if (dirty) queue[qn + __popc(bal & lt_lanes)] = uint16_t(code);
            qn += __popc(bal);
        }
        __syncwarp();
        // 2. test and lower them
        bool chg = false;
        for (int k = lane; k < qn; k += 32) {
            const int code = queue[k];
            const int sr = code >> 6, q = code & 63, sb = 8 * q;
            uint32_t vm = 0;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                vm |= (unsigned(sb + px + 2 * kk - slo) <= unsigned(shi - slo) ? 1u : 0u) << (8 * kk);
            const bool inside = unsigned(sr - V.hr) < unsigned(V.th) && sb >= V.pad && sb < V.pad + V.tw;
            const uint32_t in = inside ? vm : 0u;
            ntest += __popc(in);
            uint32_t moved, aff;  // (this engine marks whole cells: aff is not used)
            T *rb = tile + sr * bw + sb;
            if (sizeof(T) == 1 && !(V.rule & 4))  // u8 under (8,4): four points at once
                moved = item_u8(reinterpret_cast<const uint8_t *>(rb - bw), reinterpret_cast<uint8_t *>(rb),
                                reinterpret_cast<const uint8_t *>(rb + bw), px, vm, in, V.lam, V.rule,
                                nlow, aff);
            else if (sizeof(T) == 2 && !(V.rule & 4))  // u16 under (8,4): four points in 16-bit lanes
                moved = item_u16(reinterpret_cast<const uint16_t *>(rb - bw), reinterpret_cast<uint16_t *>(rb),
                                 reinterpret_cast<const uint16_t *>(rb + bw), px, vm, in, ~0u, V.lam,
                                 V.rule, nlow, aff);
            else
                moved = item_table<T>(rb - bw, rb, rb + bw, px, vm, in, tabs + ((V.rule & 4) ? kTabOffset48 : 0), V.lam,
                                      V.rule, nlow);
            if (moved) {
                cells[((sr >> 1) + 1) * ccols + q + 1] = rel;
                if (moved & in) chg = true;
            }
        }
        if (__any_sync(0xffffffffu, chg)) chg_j = j;
        __syncwarp();
    }
}

// Store the tile interior (clipped to the image) to `dst`; 16 bytes of left pad.
__device__ void tile_store(const uint8_t *tile, int bw_bytes, int es, const Visit &V, char *dst, size_t pitch)
{
    const int lane = threadIdx.x & 31;
    const int cw = min(V.tw, V.w - V.x0) * es, ch = min(V.th, V.h - V.y0);
    const int rowb = V.tw * es;
    char *base = dst + size_t(V.y0) * pitch + size_t(V.x0) * es;
    const uint8_t *src = tile + V.hr * bw_bytes + 16;
    if (cw == rowb) {
        const int vpr = rowb / 16;
        const uint32_t Mv = div_magic(vpr);
        for (int v = lane; v < ch * vpr; v += 32) {
            const int row = div_small(v, vpr, Mv), col = v - row * vpr;
            *reinterpret_cast<uint4 *>(base + size_t(row) * pitch + col * 16) =
                *reinterpret_cast<const uint4 *>(src + row * bw_bytes + col * 16);
        }
    } else {
        const uint32_t Mc = div_magic(cw);
        for (int e = lane; e < ch * cw; e += 32) {
            const int row = div_small(e, cw, Mc), col = e - row * cw;
            base[size_t(row) * pitch + col] = char(src[row * bw_bytes + col]);
        }
    }
}

__device__ __forceinline__ void decode(const EngineArgs &P, bool full, const unsigned *L, unsigned i, int &img,
                                       int &tx, int &ty)
{
    const int gt = full ? int(i) : int(__ldcg(L + i));  // written by other blocks: bypass L1
    img = find_image(P.imgs, P.n_imgs, gt);
    const ImgDesc &D = P.imgs[img];
    const int local = gt - D.tile_base;
    ty = local / D.tiles_x;
    tx = local - ty * D.tiles_x;
}

constexpr int kSmemTabs = 4 * kTabWords;  // point tables of (8,4) and (4,8), 256 x u32 each

__global__ void __launch_bounds__(kThreads, 2) k_engine(EngineArgs P)
{
    extern __shared__ __align__(128) uint8_t smem_raw[];
    // TMA destinations want 128-byte aligned shared addresses
    uint8_t *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    uint32_t *tabs = reinterpret_cast<uint32_t *>(smem);
    __shared__ int s_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const WarpLayout WL = P.wl;
    uint8_t *wbase = smem + kSmemTabs + warp * WL.bytes;
    uint8_t *tile = wbase;
    int32_t *cells = reinterpret_cast<int32_t *>(wbase + WL.cell_off);
    uint16_t *queue = reinterpret_cast<uint16_t *>(wbase + WL.queue_off);
    const uint32_t bar = smem_u32(wbase + WL.bar_off);

    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        tabs[i] = d_point_table.v[i];
        tabs[kTabOffset48 + i] = d_point_table48.v[i];
    }
    if (lane == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    uint32_t parity = 0;
    long long g0 = P.start_phase;
    const int H = P.halo, HR = P.hr;
    const unsigned nwarps = gridDim.x * kWarps;
    // consecutive items go to different blocks first, so that a step with few
    // tiles spreads them over the SMs instead of stacking them on one
    const unsigned gw = warp * gridDim.x + blockIdx.x;
    const uint32_t Mcc = div_magic(WL.ccols);
    for (int s = 0;; ++s) {
        const long long done = g0 - P.start_phase;
        const int Hs = (P.max_phases >= 0 && P.max_phases - done < H) ? int(P.max_phases - done) : H;
        const bool full = done <= 3;
        const unsigned count = full ? unsigned(P.total_tiles)
                                    : *reinterpret_cast<volatile unsigned *>(&P.ctl->list_count[s % 3]);
        const unsigned *L = P.lists + size_t(s % 3) * P.total_tiles;
        unsigned *Lnext = P.lists + size_t((s + 1) % 3) * P.total_tiles;
        if (blockIdx.x == 0 && threadIdx.x == 0) {  // counters of step s + 2, last used in step s - 1
            P.ctl->list_count[(s + 2) % 3] = 0;
            P.ctl->next_item[(s + 2) % 3] = 0;
        }
        const int src = s & 1;
        bool failed = false;
        // Every warp takes item gw first, then claims further items one at a time from the step's counter,
        // so that warps that drew light tiles take more of them and the step ends with the grid together.
        for (unsigned i = gw; i < count;) {
            int img, tx, ty;
            decode(P, full, L, i, img, tx, ty);
            const ImgDesc &D = P.imgs[img];
            Visit V;
            V.w = D.w;
            V.h = D.h;
            V.lam = D.lam;
            V.rule = P.rule | (D.adj << 2);  // F^- reading, operator, adjacency pair
            V.tw = P.tw;
            V.th = P.th;
            V.H = H;
            V.Hs = Hs;
            V.hr = HR;
            V.g0 = g0;
            V.start = P.start_phase;
            V.x0 = tx * P.tw;
            V.y0 = ty * P.th;
            const int u16 = D.dtype == THIN_U16;
            const int es = u16 ? 2 : 1;
            V.pad = 16 / es;
            const int bw = P.tw + 2 * V.pad;  // elements per shared row
            const size_t pitch = D.pitch;
            char *dst = reinterpret_cast<char *>(D.buf[src ^ 1]);
            if (lane == 0) {
                const uint32_t bytes = uint32_t(bw * es * (P.th + 2 * HR));
                tma_load_2d(smem_u32(tile), &D.map[src], V.x0 - V.pad, V.y0 - HR, bar, bytes);
            }
            // stamps of the region (overlaps the load); the border ring never changes
            {
                const int32_t *gc = reinterpret_cast<const int32_t *>(D.cells);
                const int cx0 = (V.x0 - V.pad) / 8 - 1, cy0 = (V.y0 - HR) / 2 - 1;
                const int n = WL.ccols * WL.crows;
#pragma unroll 4
                for (int e = lane; e < n; e += 32) {
                    const int cy = div_small(e, WL.ccols, Mcc), cx = e - cy * WL.ccols;
                    const int gx = cx0 + cx, gy = cy0 + cy;
                    const bool ring = cx == 0 || cy == 0 || cx == WL.ccols - 1 || cy == WL.crows - 1;
                    cells[e] = (!ring && gx >= 0 && gy >= 0 && gx < D.cells_x && gy < D.cells_y)
                                   ? __ldcg(gc + size_t(gy) * D.cells_x + gx)
                                   : kNever;
                }
            }
            const bool ok = mbar_wait(bar, parity, P.timeout_ns);
            parity ^= 1u;
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) {
                    atomicCAS(&P.ctl->error, 0, THIN_ERR_TIMEOUT);
                    mbar_wait(bar, parity ^ 1u, P.timeout_ns);  // let the load in flight land (bounded)
                }
                failed = true;
                break;
            }
            __syncwarp();
            int nlow = 0, chg_j = -1, ntest = 0;
            if (u16)
                visit_phases<uint16_t>(reinterpret_cast<uint16_t *>(tile), bw, cells, WL.ccols, queue, V, tabs, nlow,
                                       chg_j, ntest);
            else
                visit_phases<uint8_t>(tile, bw, cells, WL.ccols, queue, V, tabs, nlow, chg_j, ntest);
            tile_store(tile, bw * es, es, V, dst, pitch);
            // stamps of the interior cells back to the image's stamp grid
            {
                int32_t *gc = reinterpret_cast<int32_t *>(D.cells);
                const int icx = V.tw / 8, icy = V.th / 2;
                const int cxa = V.x0 / 8, cya = V.y0 / 2;
                const int ox = V.pad / 8 + 1, oy = HR / 2 + 1;
                const uint32_t Mi = div_magic(icx);
#pragma unroll 4
                for (int e = lane; e < icx * icy; e += 32) {
                    const int cy = div_small(e, icx, Mi), cx = e - cy * icx;
                    const int gx = cxa + cx, gy = cya + cy;
                    if (gx < D.cells_x && gy < D.cells_y)
                        __stcg(gc + size_t(gy) * D.cells_x + gx, cells[(oy + cy) * WL.ccols + ox + cx]);
                }
            }
            nlow = __reduce_add_sync(0xffffffffu, nlow);
            ntest = __reduce_add_sync(0xffffffffu, ntest);
            const int maxj = __reduce_max_sync(0xffffffffu, chg_j);
            // order this warp's generic shared and global writes before later TMA traffic
            asm volatile("fence.proxy.async;" ::: "memory");
            __syncwarp();
            if (lane < 9 && maxj >= 0) {
                const int dx = lane % 3 - 1, dy = lane / 3 - 1;
                const bool self = dx == 0 && dy == 0;
                const bool late = maxj >= Hs - 3;
                const int ntx = tx + dx, nty = ty + dy;
                if ((self || late) && ntx >= 0 && ntx < D.tiles_x && nty >= 0 && nty < D.tiles_y) {
                    const int gt = D.tile_base + nty * D.tiles_x + ntx;
                    if (atomicMax(&P.listed[gt], s + 1) < s + 1) {
                        const unsigned pos = atomicAdd(&P.ctl->list_count[(s + 1) % 3], 1u);
                        Lnext[pos] = unsigned(gt);
                        atomicMax(&P.st[img].last_listed, s + 1);
                    }
                }
            }
            if (lane == 0) {
                if (nlow) atomicAdd(&P.st[img].lowered, (unsigned long long)nlow);
                if (maxj >= 0) atomicMax(&P.st[img].last_change, g0 + maxj);
                atomicAdd(&P.st[img].tiles_visited, 1ull);
                atomicAdd(&P.st[img].tested, (unsigned long long)ntest);
                atomicMax(&P.st[img].last_step, s);
            }
            unsigned nxt = 0;
            if (lane == 0) nxt = nwarps + atomicAdd(&P.ctl->next_item[s % 3], 1u);
            i = __shfl_sync(0xffffffffu, nxt, 0);
        }
        if (__syncthreads_or(failed)) {
            if (threadIdx.x == 0) atomicCAS(&P.ctl->error, 0, THIN_ERR_TIMEOUT);
            return;
        }
        const bool skip = P.debug == 1 && blockIdx.x == 0 && s == 0;
        if (!grid_barrier(P.ctl, gridDim.x, P.timeout_ns, skip, &s_flag)) return;
        g0 += Hs;
        const long long ran = g0 - P.start_phase;
        const unsigned next = *reinterpret_cast<volatile unsigned *>(&P.ctl->list_count[(s + 1) % 3]);
        const bool stop = (P.max_phases >= 0 && ran >= P.max_phases) || (ran > 3 && next == 0);
        if (stop) {
            if (blockIdx.x == 0 && threadIdx.x == 0) P.ctl->steps = s + 1;
            return;
        }
    }
}

// Copies each image's final buffer to the caller's image where they differ.
__global__ void k_copy_out(const ImgDesc *imgs, const ImgStat *st, int n)
{
    const int k = blockIdx.y;
    if (k >= n) return;
    const ImgDesc &D = imgs[k];
    const ImgStat &S = st[k];
    const bool converged = S.last_listed <= S.last_step;
    const int fin = converged ? 0 : ((S.last_step + 1) & 1);
    const char *src = reinterpret_cast<const char *>(D.buf[fin]);
    char *dst = reinterpret_cast<char *>(D.user);
    if (src == dst) return;
    const size_t rowb = size_t(D.w) * (D.dtype == THIN_U16 ? 2 : 1);
    const size_t total = rowb * size_t(D.h);
    for (size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += size_t(gridDim.x) * blockDim.x) {
        const size_t r = e / rowb, c = e - r * rowb;
        dst[r * D.user_pitch + c] = src[r * D.pitch + c];
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Shared-memory layout of one warp for tiles tw x th and halo rows hr.  The
// tile buffer fits the widest element present; the stamp grid and the queue
// fit u8 geometry (16 pad elements either side), which is the wider in cells.
WarpLayout warp_layout(int tw, int th, int hr, bool any16)
{
    WarpLayout L;
    const int bw_bytes = any16 ? (tw + 16) * 2 : tw + 32;
    const int cols8 = (tw + 32) / 8;  // cells per shared row of a u8 tile (u16: fewer)
    const int rows = th + 2 * hr;
    L.tile_bytes = int(align_up(size_t(bw_bytes) * rows + 16, 16));
    L.ccols = cols8 + 2;
    L.crows = rows / 2 + 2;
    L.cell_off = L.tile_bytes;
    const int max_items = (rows / 2 + 1) * (cols8 + 1);
    L.queue_off = int(align_up(size_t(L.cell_off) + 4 * size_t(L.ccols) * L.crows, 16));
    L.bar_off = int(align_up(size_t(L.queue_off) + 2 * size_t(max_items), 16));
    L.bytes = int(align_up(size_t(L.bar_off) + 16, 128));
    return L;
}

}  // namespace

void tiled_defaults(int dtype, int *tw, int *th, int *halo)
{
    *tw = 64;
    *th = 32;
    *halo = dtype == THIN_U16 ? 8 : 8;
}

// A tiled launch prepared on the host: layout, tensor maps and pristine
// stats/control words uploaded into one device allocation.
struct TiledPrepared {
    int n = 0, H = 0, grid = 0, smem = 0;
    bool async_alloc = true;
    char *base = nullptr;
    size_t o_stat = 0, o_ctl = 0, o_stat0 = 0, o_ctl0 = 0, o_listed = 0, o_cells = 0, cells_bytes = 0;
    int total_tiles = 0;
    std::vector<JobSpec> jobs;
    std::vector<ImgDesc> descs;
    EngineArgs P;
};

int tiled_prepare(const JobSpec *jobs, int n, const thin_options &opt, cudaStream_t stream, bool async_alloc,
                  TiledPrepared **out, int max_grid)
{
    *out = nullptr;
    bool any16 = false;
    for (int k = 0; k < n; ++k) any16 |= jobs[k].dtype == THIN_U16;
    int tw = opt.tile_w, th = opt.tile_h, H = opt.halo;
    {
        int dw, dh, dH;
        tiled_defaults(any16 ? THIN_U16 : THIN_U8, &dw, &dh, &dH);
        if (!tw) tw = dw;
        if (!th) th = dh;
        if (!H) H = dH;
    }
    const int max_halo = any16 ? 8 : 16;  // the 16-byte left pad holds the halo columns
    if (H < kMinHalo || H > max_halo || tw < 16 || tw > 224 || tw % 16 || th < 8 || th % 2 ||
        std::min(tw, th) < H + 1)
        return THIN_ERR_ARG;
    const int HR = H + (H & 1);
    if (th + 2 * HR > 256) return THIN_ERR_ARG;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return THIN_ERR_CUDA;

    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);

    TiledPrepared *T = new TiledPrepared;
    T->n = n;
    T->H = H;
    T->async_alloc = async_alloc;
    T->jobs.assign(jobs, jobs + n);
    // ---- layout of one scratch allocation
    std::vector<ImgDesc> &descs = T->descs;
    descs.resize(n);
    std::vector<size_t> buf_off(n), cpy_off(n), cell_off(n);
    size_t off = 0;
    const size_t o_desc = off;
    off = align_up(off + sizeof(ImgDesc) * n, 256);
    T->o_stat = off;
    off = align_up(off + sizeof(ImgStat) * n, 256);
    T->o_stat0 = off;
    off = align_up(off + sizeof(ImgStat) * n, 256);
    T->o_ctl = off;
    off = align_up(off + sizeof(Ctl), 256);
    T->o_ctl0 = off;
    off = align_up(off + sizeof(Ctl), 256);
    int total_tiles = 0;
    for (int k = 0; k < n; ++k) {
        const JobSpec &J = jobs[k];
        ImgDesc &D = descs[k];
        std::memset(&D, 0, sizeof D);
        D.w = J.w;
        D.h = J.h;
        D.dtype = J.dtype;
        D.lam = J.lam;
        D.adj = J.adj;
        D.tiles_x = (J.w + tw - 1) / tw;
        D.tiles_y = (J.h + th - 1) / th;
        D.tile_base = total_tiles;
        D.cells_x = (J.w + 7) / 8;
        D.cells_y = (J.h + 1) / 2;
        total_tiles += D.tiles_x * D.tiles_y;
        const size_t es = elem_size(J.dtype);
        const bool aligned = (reinterpret_cast<uintptr_t>(J.img) % 16 == 0) && (J.pitch % 16 == 0);
        D.copy_in = aligned ? 0 : 1;
        D.pitch = aligned ? J.pitch : align_up(size_t(J.w) * es, 128);
        D.user = reinterpret_cast<unsigned long long>(J.img);
        D.user_pitch = J.pitch;
        buf_off[k] = off;
        off = align_up(off + D.pitch * J.h, 256);
        cpy_off[k] = 0;
        if (D.copy_in) {
            cpy_off[k] = off;
            off = align_up(off + D.pitch * J.h, 256);
        }
    }
    T->o_cells = off;
    for (int k = 0; k < n; ++k) {
        cell_off[k] = off;
        off = align_up(off + sizeof(int32_t) * size_t(descs[k].cells_x) * descs[k].cells_y, 256);
    }
    T->cells_bytes = off - T->o_cells;
    T->o_listed = off;
    off = align_up(off + sizeof(int) * total_tiles, 256);
    const size_t o_lists = off;
    off = align_up(off + sizeof(unsigned) * 3 * size_t(total_tiles), 256);
    const size_t total_bytes = off;
    T->total_tiles = total_tiles;

    cudaError_t e = async_alloc ? cudaMallocAsync(reinterpret_cast<void **>(&T->base), total_bytes, stream)
                                : cudaMalloc(reinterpret_cast<void **>(&T->base), total_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        T->base = nullptr;
        delete T;
        return THIN_ERR_OOM;
    }
    char *base = T->base;
    for (int k = 0; k < n; ++k) {
        ImgDesc &D = descs[k];
        const JobSpec &J = jobs[k];
        void *b0 = D.copy_in ? static_cast<void *>(base + cpy_off[k]) : J.img;
        void *b1 = base + buf_off[k];
        D.buf[0] = reinterpret_cast<unsigned long long>(b0);
        D.buf[1] = reinterpret_cast<unsigned long long>(b1);
        D.cells = reinterpret_cast<unsigned long long>(base + cell_off[k]);
        const int pad = J.dtype == THIN_U16 ? 8 : 16;
        const cuuint64_t gdim[2] = {cuuint64_t(J.w), cuuint64_t(J.h)};
        const cuuint64_t gstr[1] = {cuuint64_t(D.pitch)};
        const cuuint32_t box[2] = {cuuint32_t(tw + 2 * pad), cuuint32_t(th + 2 * HR)};
        const cuuint32_t est[2] = {1, 1};
        for (int q = 0; q < 2; ++q) {
            void *bp = q ? b1 : b0;
            CUresult r = enc(&D.map[q], J.dtype == THIN_U16 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8,
                             2, bp, gdim, gstr, box, est, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) {
                tiled_release(T, stream);
                return THIN_ERR_ARG;
            }
        }
    }
    std::vector<ImgStat> st0(n);
    for (auto &x : st0) {
        x.lowered = 0;
        x.tiles_visited = 0;
        x.tested = 0;
        x.last_change = -1;
        x.last_step = -1;
        x.last_listed = 0;
    }
    Ctl ctl0;
    std::memset(&ctl0, 0, sizeof ctl0);
    e = cudaMemcpyAsync(base + o_desc, descs.data(), sizeof(ImgDesc) * n, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + T->o_stat0, st0.data(), sizeof(ImgStat) * n, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + T->o_ctl0, &ctl0, sizeof ctl0, cudaMemcpyHostToDevice, stream);

    EngineArgs &P = T->P;
    std::memset(&P, 0, sizeof P);
    P.imgs = reinterpret_cast<const ImgDesc *>(base + o_desc);
    P.st = reinterpret_cast<ImgStat *>(base + T->o_stat);
    P.listed = reinterpret_cast<int *>(base + T->o_listed);
    P.lists = reinterpret_cast<unsigned *>(base + o_lists);
    P.ctl = reinterpret_cast<Ctl *>(base + T->o_ctl);
    P.n_imgs = n;
    P.total_tiles = total_tiles;
    P.tw = tw;
    P.th = th;
    P.halo = H;
    P.hr = HR;
    P.rule = test_mode(opt);  // F^- reading and operator
    P.start_phase = opt.start_phase;
    P.max_phases = opt.max_phases;
    P.timeout_ns = 2000000000ull;
    if (const char *t = std::getenv("THIN_TIMEOUT_NS")) P.timeout_ns = std::strtoull(t, nullptr, 10);
    P.debug = opt.reserved;
    P.wl = warp_layout(tw, th, HR, any16);
    T->smem = 128 + kSmemTabs + kWarps * P.wl.bytes;
    {
        int optin = 0;
        cudaFuncAttributes fa;
        if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
            cudaFuncGetAttributes(&fa, reinterpret_cast<const void *>(k_engine)) == cudaSuccess &&
            size_t(T->smem) + fa.sharedSizeBytes > size_t(optin)) {
            tiled_release(T, stream);
            return THIN_ERR_ARG;  // this tile shape and halo do not fit one block's shared memory
        }
    }

    if (e == cudaSuccess) e = allow_max_dynamic_smem(reinterpret_cast<const void *>(k_engine));
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_engine, kThreads, T->smem);
    if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
    T->grid = std::max(1, std::min(sms * per_sm, (total_tiles + kWarps - 1) / kWarps));
    if (max_grid > 0) T->grid = std::min(T->grid, max_grid);
    if (opt.reserved == 1) T->grid = std::max(T->grid, std::min(2, sms * per_sm));
    if (e != cudaSuccess) {
        tiled_release(T, stream);
        return cuda_status(e);
    }
    *out = T;
    return THIN_OK;
}

// Copies unaligned images in, resets the per-run state, launches the engine
// and the copy-out: device work only, so it can be captured in a CUDA graph.
cudaError_t tiled_enqueue(const TiledPrepared *T, cudaStream_t stream)
{
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < T->n && e == cudaSuccess; ++k) {
        const ImgDesc &D = T->descs[k];
        const JobSpec &J = T->jobs[k];
        if (D.copy_in)
            e = cudaMemcpy2DAsync(reinterpret_cast<void *>(D.buf[0]), D.pitch, J.img, J.pitch,
                                  size_t(J.w) * elem_size(J.dtype), J.h, cudaMemcpyDeviceToDevice, stream);
    }
    char *base = T->base;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + T->o_stat, base + T->o_stat0, sizeof(ImgStat) * T->n, cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + T->o_ctl, base + T->o_ctl0, sizeof(Ctl), cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + T->o_listed, 0xff, sizeof(int) * T->total_tiles, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + T->o_cells, 0, T->cells_bytes, stream);  // every cell: changed at the first phase
    if (e == cudaSuccess) {
        void *args[] = {const_cast<EngineArgs *>(&T->P)};
        e = cudaLaunchCooperativeKernel(reinterpret_cast<void *>(k_engine), dim3(T->grid), dim3(kThreads), args, T->smem,
                                        stream);
    }
    if (e == cudaSuccess) {
        k_copy_out<<<dim3(64, T->n), 256, 0, stream>>>(T->P.imgs, T->P.st, T->n);
        e = cudaGetLastError();
    }
    return e;
}

int tiled_collect(const TiledPrepared *T, const thin_options &opt, cudaStream_t stream, thin_stats *out)
{
    const int n = T->n;
    std::vector<ImgStat> st(n);
    Ctl ctl;
    cudaError_t e = cudaMemcpyAsync(st.data(), T->P.st, sizeof(ImgStat) * n, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ctl, T->P.ctl, sizeof ctl, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_status(e);
    int rc = THIN_OK;
    for (int k = 0; k < n; ++k) {
        const ImgStat &S = st[k];
        thin_stats &o = out[k];
        std::memset(&o, 0, sizeof o);
        const long long steps = S.last_step + 1;
        long long phases = steps * T->H;
        if (opt.max_phases >= 0) phases = std::min<long long>(phases, opt.max_phases);
        o.converged = (S.last_listed <= S.last_step && ctl.error == 0) ? 1 : 0;
        o.status = ctl.error ? ctl.error : (o.converged ? THIN_OK : THIN_ERR_NOT_CONVERGED);
        o.phases = phases;
        o.lowered = (int64_t)S.lowered;
        o.last_change_phase = S.last_change;
        o.end_phase = opt.start_phase + phases;
        o.tiles_visited = (int64_t)S.tiles_visited;
        o.tested = (int64_t)S.tested;
        o.steps = steps;
        if (o.status != THIN_OK && rc == THIN_OK) rc = o.status;
    }
    return rc;
}

void tiled_release(TiledPrepared *T, cudaStream_t stream)
{
    if (!T) return;
    if (T->base) {
        if (T->async_alloc) cudaFreeAsync(T->base, stream);
        else cudaFree(T->base);
    }
    delete T;
}

int tiled_run(const JobSpec *jobs, int n, const thin_options &opt, cudaStream_t stream, thin_stats *out)
{
    if (n <= 0) return THIN_OK;
    if (opt.max_phases == 0) {  // nothing may run: every image stays as it is, unconverged
        if (out)
            for (int k = 0; k < n; ++k) {
                std::memset(&out[k], 0, sizeof out[k]);
                out[k].status = THIN_ERR_NOT_CONVERGED;
                out[k].last_change_phase = -1;
                out[k].end_phase = opt.start_phase;
            }
        return THIN_ERR_NOT_CONVERGED;
    }
    TiledPrepared *T = nullptr;
    int rc = tiled_prepare(jobs, n, opt, stream, true, &T);
    if (rc != THIN_OK) return rc;
    const cudaError_t e = tiled_enqueue(T, stream);
    if (e != cudaSuccess) rc = cuda_status(e);
    else if (out) rc = tiled_collect(T, opt, stream, out);
    tiled_release(T, stream);
    return rc;
}

}  // namespace thin

// ---------------------------------------------------------------------------
// Allocation-free entry point.
//
// Some callers cannot allocate device memory at the moment they want to thin
// an image: an application that hands all device memory to its own allocator
// at start-up (a further cudaMalloc would fail or eat into that budget), or a
// loop with a fixed time budget that may not call into the allocator, which
// can have to map new memory or wait for the device.  thin_run_noalloc serves
// them with the tiled engine and no allocation at all: its scratch (the
// second ping-pong buffer, the change stamps, the worklists and the control
// words) lives in one fixed array in device memory that the library declares
// at file scope.  Every GPU that loads the library holds the array until the
// process exits.
static __device__ __align__(256) unsigned char g_thin_noalloc_scratch[THIN_NOALLOC_SCRATCH_BYTES];

namespace thin {
namespace {

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

struct NoallocSlot {
    unsigned long long ctx_id = 0;  // context the address belongs to (0: unknown)
    void *base = nullptr;
};
std::mutex g_noalloc_mu;
NoallocSlot g_noalloc_slot[256];

// Identity of the calling thread's current context, 0 if it cannot be had.
unsigned long long current_context_id()
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(p);
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(p);
    });
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&c) == CUDA_SUCCESS && c && get_id(c, &id) == CUDA_SUCCESS) return id;
    return 0;
}

// Device address of the scratch array on the current device (in host code the
// array's name is only a host-side stand-in).  Looked up at the first call on
// a device, and again only if the device's context has been created anew
// since (after cudaDeviceReset the array lives at a new address).
cudaError_t noalloc_scratch(void **base)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoallocSlot &S = g_noalloc_slot[dev];
    const unsigned long long id = current_context_id();
    if (!S.base || id == 0 || id != S.ctx_id) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_thin_noalloc_scratch);
        if (e != cudaSuccess) return e;
        S.base = p;
        S.ctx_id = current_context_id();  // the lookup makes the context current if it was not
    }
    *base = S.base;
    return cudaSuccess;
}

// The tiled engine on one image, with every piece of scratch carved from the
// fixed array.  Same kernels, launch and result as tiled_run.
int tiled_run_noalloc(const JobSpec &J, const thin_options &opt, cudaStream_t stream, thin_stats *out)
{
    if (opt.max_phases == 0) {
        if (out) {
            std::memset(out, 0, sizeof *out);
            out->status = THIN_ERR_NOT_CONVERGED;
            out->last_change_phase = -1;
            out->end_phase = opt.start_phase;
        }
        return THIN_ERR_NOT_CONVERGED;
    }
    const bool is16 = J.dtype == THIN_U16;
    int tw = opt.tile_w, th = opt.tile_h, H = opt.halo;
    {
        int dw, dh, dH;
        tiled_defaults(J.dtype, &dw, &dh, &dH);
        if (!tw) tw = dw;
        if (!th) th = dh;
        if (!H) H = dH;
    }
    const int max_halo = is16 ? 8 : 16;
    if (H < kMinHalo || H > max_halo || tw < 16 || tw > 224 || tw % 16 || th < 8 || th % 2 ||
        std::min(tw, th) < H + 1)
        return THIN_ERR_ARG;
    const int HR = H + (H & 1);
    if (th + 2 * HR > 256) return THIN_ERR_ARG;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return THIN_ERR_CUDA;

    ImgDesc D;
    std::memset(&D, 0, sizeof D);
    D.w = J.w;
    D.h = J.h;
    D.dtype = J.dtype;
    D.lam = J.lam;
    D.adj = J.adj;
    D.tiles_x = (J.w + tw - 1) / tw;
    D.tiles_y = (J.h + th - 1) / th;
    D.tile_base = 0;
    D.cells_x = (J.w + 7) / 8;
    D.cells_y = (J.h + 1) / 2;
    const int total_tiles = D.tiles_x * D.tiles_y;
    const size_t es = elem_size(J.dtype);
    const bool aligned = (reinterpret_cast<uintptr_t>(J.img) % 16 == 0) && (J.pitch % 16 == 0);
    D.copy_in = aligned ? 0 : 1;
    D.pitch = aligned ? J.pitch : align_up(size_t(J.w) * es, 128);
    D.user = reinterpret_cast<unsigned long long>(J.img);
    D.user_pitch = J.pitch;

    // layout inside the fixed array (same pieces as tiled_run, one image)
    size_t off = 0;
    const size_t o_desc = off;
    off = align_up(off + sizeof(ImgDesc), 256);
    const size_t o_stat = off;
    off = align_up(off + sizeof(ImgStat), 256);
    const size_t o_ctl = off;
    off = align_up(off + sizeof(Ctl), 256);
    const size_t o_buf = off;
    off = align_up(off + D.pitch * J.h, 256);
    const size_t o_cpy = off;
    if (D.copy_in) off = align_up(off + D.pitch * J.h, 256);
    const size_t o_cells = off;
    const size_t cells_bytes = sizeof(int32_t) * size_t(D.cells_x) * D.cells_y;
    off = align_up(off + cells_bytes, 256);
    const size_t o_listed = off;
    off = align_up(off + sizeof(int) * total_tiles, 256);
    const size_t o_lists = off;
    off = align_up(off + sizeof(unsigned) * 3 * size_t(total_tiles), 256);
    if (off > THIN_NOALLOC_SCRATCH_BYTES) return THIN_ERR_TOO_LARGE;

    char *base = nullptr;
    cudaError_t e = noalloc_scratch(reinterpret_cast<void **>(&base));
    if (e != cudaSuccess) return cuda_status(e);

    void *b0 = D.copy_in ? static_cast<void *>(base + o_cpy) : J.img;
    void *b1 = base + o_buf;
    if (D.copy_in)
        e = cudaMemcpy2DAsync(b0, D.pitch, J.img, J.pitch, size_t(J.w) * es, J.h, cudaMemcpyDeviceToDevice, stream);
    D.buf[0] = reinterpret_cast<unsigned long long>(b0);
    D.buf[1] = reinterpret_cast<unsigned long long>(b1);
    D.cells = reinterpret_cast<unsigned long long>(base + o_cells);
    {
        const int pad = is16 ? 8 : 16;
        const cuuint64_t gdim[2] = {cuuint64_t(J.w), cuuint64_t(J.h)};
        const cuuint64_t gstr[1] = {cuuint64_t(D.pitch)};
        const cuuint32_t box[2] = {cuuint32_t(tw + 2 * pad), cuuint32_t(th + 2 * HR)};
        const cuuint32_t est[2] = {1, 1};
        for (int q = 0; q < 2; ++q) {
            CUresult r = enc(&D.map[q], is16 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                             q ? b1 : b0, gdim, gstr, box, est, CU_TENSOR_MAP_INTERLEAVE_NONE,
                             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return THIN_ERR_ARG;
        }
    }
    // the array keeps the previous call's contents: set everything the engine reads
    ImgStat st0;
    st0.lowered = 0;
    st0.tiles_visited = 0;
    st0.tested = 0;
    st0.last_change = -1;
    st0.last_step = -1;
    st0.last_listed = 0;
    Ctl ctl0;
    std::memset(&ctl0, 0, sizeof ctl0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_desc, &D, sizeof D, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_stat, &st0, sizeof st0, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_ctl, &ctl0, sizeof ctl0, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_listed, 0xff, sizeof(int) * total_tiles, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_cells, 0, cells_bytes, stream);

    EngineArgs P;
    std::memset(&P, 0, sizeof P);
    P.imgs = reinterpret_cast<const ImgDesc *>(base + o_desc);
    P.st = reinterpret_cast<ImgStat *>(base + o_stat);
    P.listed = reinterpret_cast<int *>(base + o_listed);
    P.lists = reinterpret_cast<unsigned *>(base + o_lists);
    P.ctl = reinterpret_cast<Ctl *>(base + o_ctl);
    P.n_imgs = 1;
    P.total_tiles = total_tiles;
    P.tw = tw;
    P.th = th;
    P.halo = H;
    P.hr = HR;
    P.rule = test_mode(opt);  // F^- reading and operator
    P.start_phase = opt.start_phase;
    P.max_phases = opt.max_phases;
    P.timeout_ns = 2000000000ull;
    if (const char *t = std::getenv("THIN_TIMEOUT_NS")) P.timeout_ns = std::strtoull(t, nullptr, 10);
    P.debug = 0;
    P.wl = warp_layout(tw, th, HR, is16);
    const int smem = 128 + kSmemTabs + kWarps * P.wl.bytes;

    int dev = 0, sms = 0, per_sm = 0, optin = 0;
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, reinterpret_cast<const void *>(k_engine));
    if (e == cudaSuccess && size_t(smem) + fa.sharedSizeBytes > size_t(optin)) return THIN_ERR_ARG;
    if (e == cudaSuccess) e = allow_max_dynamic_smem(reinterpret_cast<const void *>(k_engine));
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_engine, kThreads, smem);
    if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
    const int grid = std::max(1, std::min(sms * per_sm, (total_tiles + kWarps - 1) / kWarps));
    if (e == cudaSuccess) {
        void *args[] = {&P};
        e = cudaLaunchCooperativeKernel(reinterpret_cast<void *>(k_engine), dim3(grid), dim3(kThreads), args, smem,
                                        stream);
    }
    if (e == cudaSuccess) {
        k_copy_out<<<dim3(64, 1), 256, 0, stream>>>(P.imgs, P.st, 1);
        e = cudaGetLastError();
    }
    int rc = THIN_OK;
    if (e == cudaSuccess && out) {
        ImgStat S;
        Ctl ctl;
        e = cudaMemcpyAsync(&S, P.st, sizeof S, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&ctl, P.ctl, sizeof ctl, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e == cudaSuccess) {
            std::memset(out, 0, sizeof *out);
            const long long steps = S.last_step + 1;
            long long phases = steps * H;
            if (opt.max_phases >= 0) phases = std::min<long long>(phases, opt.max_phases);
            out->converged = (S.last_listed <= S.last_step && ctl.error == 0) ? 1 : 0;
            out->status = ctl.error ? ctl.error : (out->converged ? THIN_OK : THIN_ERR_NOT_CONVERGED);
            out->phases = phases;
            out->lowered = (int64_t)S.lowered;
            out->last_change_phase = S.last_change;
            out->end_phase = opt.start_phase + phases;
            out->tiles_visited = (int64_t)S.tiles_visited;
            out->tested = (int64_t)S.tested;
            out->steps = steps;
            rc = out->status;
        }
    }
    if (e != cudaSuccess) return cuda_status(e);
    return rc;
}

}  // namespace
}  // namespace thin

extern "C" int thin_run_noalloc(void *img_dev, int w, int h, size_t pitch_bytes, thin_dtype dt, uint32_t lambda,
                                thin_adj adj, void *stream, const thin_options *opt, thin_stats *out)
{
    thin_options o;
    thin_default_options(&o);
    if (opt) o = *opt;
    if (adj != THIN_ADJ_8_4 && adj != THIN_ADJ_4_8) return THIN_ERR_ARG;
    if (o.rule != THIN_RULE_MAX && o.rule != THIN_RULE_MIN) return THIN_ERR_ARG;
    if (o.op != THIN_OP_THINNING && o.op != THIN_OP_SKELETON) return THIN_ERR_ARG;
    if (o.start_phase < 0 || o.tile_w < 0 || o.tile_h < 0 || o.halo < 0) return THIN_ERR_ARG;
    if (w < 0 || h < 0 || (dt != THIN_U8 && dt != THIN_U16)) return THIN_ERR_ARG;
    const size_t es = dt == THIN_U16 ? 2 : 1;
    if (w > 0 && h > 0) {
        if (!img_dev || pitch_bytes < size_t(w) * es) return THIN_ERR_ARG;
        if (es == 2 && ((reinterpret_cast<uintptr_t>(img_dev) & 1) || (pitch_bytes & 1))) return THIN_ERR_ARG;
    }
    if (w < 3 || h < 3) {  // empty, or no interior point: nothing to do
        if (out) {
            std::memset(out, 0, sizeof *out);
            out->converged = 1;
            out->last_change_phase = -1;
            out->end_phase = o.start_phase;
        }
        return THIN_OK;
    }
    thin::JobSpec j{img_dev, w, h, pitch_bytes, int(dt), lambda, int(adj)};
    return thin::tiled_run_noalloc(j, o, static_cast<cudaStream_t>(stream), out);
}
