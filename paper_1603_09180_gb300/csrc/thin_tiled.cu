// thin_tiled.cu -- the tiled lambda-thinning engine.
//
// One persistent cooperative launch runs the whole subfield schedule for any
// number of images.  The schedule advances in steps of H phases (temporal
// blocking).  In a step every active tile of every image is staged in shared
// memory with a halo of H pixels by a TMA 2-D tile load, advances H
// consecutive phases there (the exact region shrinks by one pixel ring per
// phase, so the TW x TH interior is exact after H phases) and is stored to the
// other buffer of a ping-pong pair.  A grid barrier separates steps.
//
// Active tiles.  Let a tile step start at global phase g0.  A point can only
// become lambda-destructible after one of its 8 neighbours changed, so at
// phase g0 every unstable point lies next to a point that changed during
// phases g0-3 .. g0-1 (every point was visited in the four phases before its
// own last visit).  Unstable points spread by at most one pixel per phase, so
// a tile none of whose 3x3 block of tiles changed in those three phases cannot
// change during the next H <= min(TW, TH) - 1 phases: it is skipped.  A tile
// that changed at all in a step is also visited in the next one, which keeps
// both ping-pong buffers equal on every skipped tile.  The first step (and
// any step starting within three phases of the first) visits every tile.
// When a step visits no tile the image is at its fixed point and both buffers
// hold it.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "thin_common.cuh"
#include "thin_internal.h"

namespace thin {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxHalo = 8;
constexpr int kMinHalo = 3;

struct ImgDesc {
    CUtensorMap map[2];          // TMA descriptors of buffer 0 and buffer 1
    unsigned long long buf[2];   // device pointers of the ping-pong pair
    unsigned long long pitch;    // row pitch of both buffers, bytes
    unsigned long long user;     // caller's image
    unsigned long long user_pitch;
    int w, h, dtype;
    unsigned lam;
    int tiles_x, tiles_y, tile_base, copy_in;
};

struct ImgStat {
    unsigned long long lowered;
    unsigned long long tiles_visited;
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
    int pad;
};

struct EngineArgs {
    const ImgDesc *imgs;
    ImgStat *st;
    int *listed;       // per tile: last step index it was appended for
    unsigned *lists;   // 3 lists of total_tiles entries each
    Ctl *ctl;
    int n_imgs;
    int total_tiles;
    int tw, th, halo, rule;
    long long start_phase;
    long long max_phases;
    unsigned long long timeout_ns;
    int buf_bytes;     // shared bytes reserved per tile buffer
    int debug;         // 1: block 0 never arrives at the first barrier (timeout test)
};

__device__ const PointTable d_tiled_table = kPointTable;

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
                __nanosleep(32);
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

// H phases of the subfield schedule on a staged tile.  Shared cell (sx, sy)
// holds image pixel (x0 - A + sx, y0 - H + sy), A = 16 bytes of elements.
template <typename T>
__device__ void tile_phases(T *tile, int bw, const ImgDesc &D, int x0, int y0, int tw, int th, int H, int Hs,
                            long long g0, const uint32_t *tab, int rule, int &nlow, int &chg_j)
{
    constexpr int A = 16 / int(sizeof(T));
    for (int j = 0; j < Hs; ++j) {
        const int p = int((g0 + j) & 3);
        const int px = p & 1, py = p >> 1;
        const int r = Hs - 1 - j;
        const int lox = max(x0 - r, 1), hix = min(x0 + tw + r - 1, D.w - 2);
        const int loy = max(y0 - r, 1), hiy = min(y0 + th + r - 1, D.h - 2);
        const int xa = lox + ((px - lox) & 1), ya = loy + ((py - loy) & 1);
        const int nx = hix >= xa ? (hix - xa) / 2 + 1 : 0;
        const int ny = hiy >= ya ? (hiy - ya) / 2 + 1 : 0;
        const int total = nx * ny;
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int k = idx / nx, i = idx - k * nx;
            const int x = xa + 2 * i, y = ya + 2 * k;
            T *q = tile + (y - y0 + H) * bw + (x - x0 + A);
            uint32_t nb[8] = {q[1], q[1 - bw], q[-bw], q[-1 - bw], q[-1], q[bw - 1], q[bw], q[bw + 1]};
            int nl = 0;
            const uint32_t c2 = lower_point(q[0], nb, tab, D.lam, rule, nl);
            if (nl) {
                q[0] = static_cast<T>(c2);
                if (x >= x0 && x < x0 + tw && y >= y0 && y < y0 + th) {
                    nlow += nl;
                    chg_j = j;
                }
            }
        }
        __syncthreads();
    }
}

// Store the tile interior (clipped to the image) to `dst`.
template <typename T>
__device__ void tile_store(const T *tile, int bw, const ImgDesc &D, char *dst, int x0, int y0, int tw, int th, int H)
{
    constexpr int A = 16 / int(sizeof(T));
    const int cw = min(tw, D.w - x0), ch = min(th, D.h - y0);
    if (cw == tw) {
        const int vpr = tw * int(sizeof(T)) / 16;
        for (int v = threadIdx.x; v < ch * vpr; v += blockDim.x) {
            const int row = v / vpr, col = v - row * vpr;
            const uint4 val = *reinterpret_cast<const uint4 *>(
                reinterpret_cast<const char *>(tile + (H + row) * bw + A) + col * 16);
            *reinterpret_cast<uint4 *>(dst + size_t(y0 + row) * D.pitch + size_t(x0) * sizeof(T) + col * 16) = val;
        }
    } else {
        for (int e = threadIdx.x; e < ch * cw; e += blockDim.x) {
            const int row = e / cw, col = e - row * cw;
            reinterpret_cast<T *>(dst + size_t(y0 + row) * D.pitch)[x0 + col] = tile[(H + row) * bw + A + col];
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

__device__ __forceinline__ void issue(const EngineArgs &P, int img, int tx, int ty, int src, uint8_t *buf,
                                      uint32_t bar)
{
    const ImgDesc &D = P.imgs[img];
    const int A = D.dtype == THIN_U16 ? 8 : 16;
    const int es = D.dtype == THIN_U16 ? 2 : 1;
    const uint32_t bytes = uint32_t((P.tw + 2 * A) * es * (P.th + 2 * P.halo));
    tma_load_2d(smem_u32(buf), &D.map[src], tx * P.tw - A, ty * P.th - P.halo, bar, bytes);
}

__global__ void __launch_bounds__(kThreads) k_engine(EngineArgs P)
{
    extern __shared__ __align__(128) uint8_t smem_raw[];
    // TMA destinations want 128-byte aligned shared addresses
    uint8_t *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    uint32_t *tab = reinterpret_cast<uint32_t *>(smem);
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(smem + 1024);
    uint8_t *bufs[2] = {smem + 1152, smem + 1152 + P.buf_bytes};
    __shared__ int s_flag, s_nlow, s_maxj;

    for (int i = threadIdx.x; i < 256; i += blockDim.x) tab[i] = d_tiled_table.v[i];
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bars[0]), 1);
        mbar_init(smem_u32(&bars[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    uint32_t ph[2] = {0, 0};
    long long g0 = P.start_phase;
    const int H = P.halo;
    for (int s = 0;; ++s) {
        const long long done = g0 - P.start_phase;
        const int Hs = (P.max_phases >= 0 && P.max_phases - done < H) ? int(P.max_phases - done) : H;
        const bool full = done <= 3;
        const unsigned count = full ? unsigned(P.total_tiles)
                                    : *reinterpret_cast<volatile unsigned *>(&P.ctl->list_count[s % 3]);
        const unsigned *L = P.lists + size_t(s % 3) * P.total_tiles;
        unsigned *Lnext = P.lists + size_t((s + 1) % 3) * P.total_tiles;
        if (blockIdx.x == 0 && threadIdx.x == 0) P.ctl->list_count[(s + 2) % 3] = 0;
        const int src = s & 1;

        int b = 0;
        unsigned i = blockIdx.x;
        int img = 0, tx = 0, ty = 0;
        if (i < count) {
            decode(P, full, L, i, img, tx, ty);
            if (threadIdx.x == 0) issue(P, img, tx, ty, src, bufs[b], smem_u32(&bars[b]));
        }
        bool failed = false;
        while (i < count) {
            const unsigned nxt = i + gridDim.x;
            int nimg = 0, ntx = 0, nty = 0;
            if (nxt < count) {
                decode(P, full, L, nxt, nimg, ntx, nty);
                if (threadIdx.x == 0) issue(P, nimg, ntx, nty, src, bufs[b ^ 1], smem_u32(&bars[b ^ 1]));
            }
            const ImgDesc &D = P.imgs[img];
            const bool ok = mbar_wait(smem_u32(&bars[b]), ph[b], P.timeout_ns);
            ph[b] ^= 1u;
            if (!__syncthreads_and(ok)) {
                if (threadIdx.x == 0) atomicCAS(&P.ctl->error, 0, THIN_ERR_TIMEOUT);
                failed = true;
                break;
            }
            if (threadIdx.x == 0) {
                s_nlow = 0;
                s_maxj = -1;
            }
            __syncthreads();
            int nlow = 0, chg_j = -1;
            const int x0 = tx * P.tw, y0 = ty * P.th;
            char *dst = reinterpret_cast<char *>(D.buf[src ^ 1]);
            if (D.dtype == THIN_U16) {
                const int bw = P.tw + 16;
                uint16_t *t16 = reinterpret_cast<uint16_t *>(bufs[b]);
                tile_phases<uint16_t>(t16, bw, D, x0, y0, P.tw, P.th, H, Hs, g0, tab, P.rule, nlow, chg_j);
                tile_store<uint16_t>(t16, bw, D, dst, x0, y0, P.tw, P.th, H);
            } else {
                const int bw = P.tw + 32;
                uint8_t *t8 = bufs[b];
                tile_phases<uint8_t>(t8, bw, D, x0, y0, P.tw, P.th, H, Hs, g0, tab, P.rule, nlow, chg_j);
                tile_store<uint8_t>(t8, bw, D, dst, x0, y0, P.tw, P.th, H);
            }
            // block reduction of the tile's lowering count and last changing phase
            for (int o = 16; o; o >>= 1) {
                nlow += __shfl_down_sync(0xffffffffu, nlow, o);
                chg_j = max(chg_j, __shfl_down_sync(0xffffffffu, chg_j, o));
            }
            if ((threadIdx.x & 31) == 0) {
                if (nlow) atomicAdd(&s_nlow, nlow);
                if (chg_j >= 0) atomicMax(&s_maxj, chg_j);
            }
            // order this tile's generic shared and global writes before later TMA traffic
            asm volatile("fence.proxy.async;" ::: "memory");
            __syncthreads();
            const int maxj = s_maxj;
            if (threadIdx.x < 9 && maxj >= 0) {
                const int dx = int(threadIdx.x % 3) - 1, dy = int(threadIdx.x / 3) - 1;
                const bool self = dx == 0 && dy == 0;
                const bool late = maxj >= Hs - 3;
                const int ntx2 = tx + dx, nty2 = ty + dy;
                if ((self || late) && ntx2 >= 0 && ntx2 < D.tiles_x && nty2 >= 0 && nty2 < D.tiles_y) {
                    const int gt = D.tile_base + nty2 * D.tiles_x + ntx2;
                    if (atomicMax(&P.listed[gt], s + 1) < s + 1) {
                        const unsigned pos = atomicAdd(&P.ctl->list_count[(s + 1) % 3], 1u);
                        Lnext[pos] = unsigned(gt);
                        atomicMax(&P.st[img].last_listed, s + 1);
                    }
                }
            }
            if (threadIdx.x == 0) {
                if (s_nlow) atomicAdd(&P.st[img].lowered, (unsigned long long)s_nlow);
                if (maxj >= 0) atomicMax(&P.st[img].last_change, g0 + maxj);
                atomicAdd(&P.st[img].tiles_visited, 1ull);
                atomicMax(&P.st[img].last_step, s);
            }
            b ^= 1;
            i = nxt;
            img = nimg;
            tx = ntx;
            ty = nty;
        }
        if (failed) {
            // let a load still in flight land before leaving (bounded)
            if (i + gridDim.x < count) mbar_wait(smem_u32(&bars[b ^ 1]), ph[b ^ 1], P.timeout_ns);
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

}  // namespace

void tiled_defaults(int dtype, int *tw, int *th, int *halo)
{
    *tw = dtype == THIN_U16 ? 64 : 64;
    *th = 64;
    *halo = 8;
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
    int tw = opt.tile_w, th = opt.tile_h, H = opt.halo;
    {
        int dw, dh, dH;
        tiled_defaults(jobs[0].dtype, &dw, &dh, &dH);
        if (!tw) tw = dw;
        if (!th) th = dh;
        if (!H) H = dH;
    }
    if (H < kMinHalo || H > kMaxHalo || tw < 16 || tw > 224 || tw % 16 || th < 8 || th + 2 * H > 256 ||
        std::min(tw, th) < H + 1)
        return THIN_ERR_ARG;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return THIN_ERR_CUDA;

    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);

    // ---- layout of one scratch allocation
    std::vector<ImgDesc> descs(n);
    std::vector<size_t> buf_off(n), cpy_off(n);
    size_t off = 0;
    const size_t o_desc = off;
    off = align_up(off + sizeof(ImgDesc) * n, 256);
    const size_t o_stat = off;
    off = align_up(off + sizeof(ImgStat) * n, 256);
    const size_t o_ctl = off;
    off = align_up(off + sizeof(Ctl), 256);
    int total_tiles = 0;
    bool any16 = false;
    for (int k = 0; k < n; ++k) {
        const JobSpec &J = jobs[k];
        ImgDesc &D = descs[k];
        std::memset(&D, 0, sizeof D);
        D.w = J.w;
        D.h = J.h;
        D.dtype = J.dtype;
        D.lam = J.lam;
        D.tiles_x = (J.w + tw - 1) / tw;
        D.tiles_y = (J.h + th - 1) / th;
        D.tile_base = total_tiles;
        total_tiles += D.tiles_x * D.tiles_y;
        any16 |= J.dtype == THIN_U16;
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
    const size_t o_listed = off;
    off = align_up(off + sizeof(int) * total_tiles, 256);
    const size_t o_lists = off;
    off = align_up(off + sizeof(unsigned) * 3 * size_t(total_tiles), 256);
    const size_t total_bytes = off;

    char *base = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void **>(&base), total_bytes, stream) != cudaSuccess) {
        cudaGetLastError();
        return THIN_ERR_OOM;
    }
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < n && e == cudaSuccess; ++k) {
        ImgDesc &D = descs[k];
        const JobSpec &J = jobs[k];
        void *b0 = D.copy_in ? static_cast<void *>(base + cpy_off[k]) : J.img;
        void *b1 = base + buf_off[k];
        if (D.copy_in)
            e = cudaMemcpy2DAsync(b0, D.pitch, J.img, J.pitch, size_t(J.w) * elem_size(J.dtype), J.h,
                                  cudaMemcpyDeviceToDevice, stream);
        D.buf[0] = reinterpret_cast<unsigned long long>(b0);
        D.buf[1] = reinterpret_cast<unsigned long long>(b1);
        const int A = J.dtype == THIN_U16 ? 8 : 16;
        const cuuint64_t gdim[2] = {cuuint64_t(J.w), cuuint64_t(J.h)};
        const cuuint64_t gstr[1] = {cuuint64_t(D.pitch)};
        const cuuint32_t box[2] = {cuuint32_t(tw + 2 * A), cuuint32_t(th + 2 * H)};
        const cuuint32_t est[2] = {1, 1};
        for (int q = 0; q < 2; ++q) {
            void *bp = q ? b1 : b0;
            CUresult r = enc(&D.map[q], J.dtype == THIN_U16 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8,
                             2, bp, gdim, gstr, box, est, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) {
                cudaFreeAsync(base, stream);
                return THIN_ERR_ARG;
            }
        }
    }
    std::vector<ImgStat> st0(n);
    for (auto &s : st0) {
        s.lowered = 0;
        s.tiles_visited = 0;
        s.last_change = -1;
        s.last_step = -1;
        s.last_listed = 0;
    }
    Ctl ctl0;
    std::memset(&ctl0, 0, sizeof ctl0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_desc, descs.data(), sizeof(ImgDesc) * n, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_stat, st0.data(), sizeof(ImgStat) * n, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_ctl, &ctl0, sizeof ctl0, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_listed, 0xff, sizeof(int) * total_tiles, stream);

    EngineArgs P;
    std::memset(&P, 0, sizeof P);
    P.imgs = reinterpret_cast<const ImgDesc *>(base + o_desc);
    P.st = reinterpret_cast<ImgStat *>(base + o_stat);
    P.listed = reinterpret_cast<int *>(base + o_listed);
    P.lists = reinterpret_cast<unsigned *>(base + o_lists);
    P.ctl = reinterpret_cast<Ctl *>(base + o_ctl);
    P.n_imgs = n;
    P.total_tiles = total_tiles;
    P.tw = tw;
    P.th = th;
    P.halo = H;
    P.rule = opt.rule;
    P.start_phase = opt.start_phase;
    P.max_phases = opt.max_phases;
    P.timeout_ns = 2000000000ull;
    if (const char *t = std::getenv("THIN_TIMEOUT_NS")) P.timeout_ns = std::strtoull(t, nullptr, 10);
    P.debug = opt.reserved;
    P.buf_bytes = int(align_up(size_t(tw + 32) * (th + 2 * H), 128));  // 32 bytes of pad = 2 x 16 B either side
    if (any16) P.buf_bytes = int(align_up(size_t(tw + 16) * 2 * (th + 2 * H), 128));
    const int smem = 128 + 1152 + 2 * P.buf_bytes;

    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_engine, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_engine, kThreads, smem);
    if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
    int grid = std::max(1, std::min(sms * per_sm, total_tiles));
    if (opt.reserved == 1) grid = std::max(grid, std::min(2, sms * per_sm));
    if (e == cudaSuccess) {
        void *args[] = {&P};
        e = cudaLaunchCooperativeKernel(reinterpret_cast<void *>(k_engine), dim3(grid), dim3(kThreads), args, smem,
                                        stream);
    }
    if (e == cudaSuccess) {
        k_copy_out<<<dim3(64, n), 256, 0, stream>>>(P.imgs, P.st, n);
        e = cudaGetLastError();
    }
    int rc = THIN_OK;
    if (e == cudaSuccess && out) {
        std::vector<ImgStat> st(n);
        Ctl ctl;
        e = cudaMemcpyAsync(st.data(), P.st, sizeof(ImgStat) * n, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&ctl, P.ctl, sizeof ctl, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e == cudaSuccess) {
            for (int k = 0; k < n; ++k) {
                const ImgStat &S = st[k];
                thin_stats &o = out[k];
                std::memset(&o, 0, sizeof o);
                const long long steps = S.last_step + 1;
                long long phases = steps * H;
                if (opt.max_phases >= 0) phases = std::min<long long>(phases, opt.max_phases);
                o.converged = (S.last_listed <= S.last_step && ctl.error == 0) ? 1 : 0;
                o.status = ctl.error ? ctl.error : (o.converged ? THIN_OK : THIN_ERR_NOT_CONVERGED);
                o.phases = phases;
                o.lowered = (int64_t)S.lowered;
                o.last_change_phase = S.last_change;
                o.end_phase = opt.start_phase + phases;
                o.tiles_visited = (int64_t)S.tiles_visited;
                o.steps = steps;
                if (o.status != THIN_OK && rc == THIN_OK) rc = o.status;
            }
        }
    }
    cudaFreeAsync(base, stream);
    if (e != cudaSuccess) return cuda_status(e);
    return rc;
}

}  // namespace thin
