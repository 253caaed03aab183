// thin_api.cu -- the C-ABI of libthin.so: argument checks, and the dispatch
// of a batch into launch groups (resident clusters by size, wide launches,
// the tiled engine) that run side by side where they can.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "thin_common.cuh"
#include "thin_internal.h"

namespace thin {

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return THIN_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? THIN_ERR_OOM : THIN_ERR_CUDA;
}

cudaError_t allow_max_dynamic_smem(const void *kernel)
{
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);  // static shared memory counts against the cap
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - int(fa.sharedSizeBytes));
    return e;
}

namespace {

int check_options(const thin_options &o)
{
    if (o.rule != THIN_RULE_MAX && o.rule != THIN_RULE_MIN) return THIN_ERR_ARG;
    if (o.op != THIN_OP_THINNING && o.op != THIN_OP_SKELETON) return THIN_ERR_ARG;
    if (o.kernel < THIN_KERNEL_AUTO || o.kernel > THIN_KERNEL_RESIDENT) return THIN_ERR_ARG;
    if (o.start_phase < 0) return THIN_ERR_ARG;
    if (o.tile_w < 0 || o.tile_h < 0 || o.halo < 0) return THIN_ERR_ARG;
    return THIN_OK;
}

// 0: valid with an interior; 1: valid, nothing to do; < 0: error code.
int check_image(const void *img, int w, int h, size_t pitch, int dt)
{
    if (w < 0 || h < 0) return THIN_ERR_ARG;
    if (dt != THIN_U8 && dt != THIN_U16) return THIN_ERR_ARG;
    if (w == 0 || h == 0) return 1;
    if (!img) return THIN_ERR_ARG;
    const size_t es = elem_size(dt);
    if (pitch < size_t(w) * es) return THIN_ERR_ARG;
    if (es == 2 && ((reinterpret_cast<uintptr_t>(img) & 1) || (pitch & 1))) return THIN_ERR_ARG;
    if (w < 3 || h < 3) return 1;
    return 0;
}

}  // namespace

// Splits validated images into launch groups: images that fit the shared
// memory of a cluster go to the resident engine, grouped by cluster size
// (AUTO, RESIDENT); the rest go to the tiled engine (AUTO, TILED).  When few
// images fit, each is spread over a wider cluster (at least 32 rows a block)
// so that more SMs work on it.
constexpr int kWideMax = 2;

int group_jobs(const std::vector<JobSpec> &specs, const thin_options &o, Grouping *G, bool allow_wide)
{
    const int n = int(specs.size());
    G->resident.clear();
    G->wide.clear();
    G->tiled.clear();
    G->nw = 16;  // warps per resident block (one block per SM measured fastest)
    std::vector<int> cls(n, 0);
    if (o.kernel == THIN_KERNEL_AUTO || o.kernel == THIN_KERNEL_RESIDENT) {
        const size_t limit = resident_smem_limit(16 / G->nw);
        for (int k = 0; k < n; ++k)
            cls[k] = resident_cluster_size(specs[k].w, specs[k].h, specs[k].dtype, limit, G->nw, nullptr, nullptr);
    }
    int eligible = 0, sms = 0, dev = 0;
    for (int k = 0; k < n; ++k) eligible += cls[k] > 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int spread = 1;
    while (eligible > 0 && spread < 8 && spread * 2 * eligible <= sms * (16 / G->nw)) spread *= 2;
    // one launch per cluster size and element size (the kernel is built for each element size)
    for (int C = 1; C <= 16; C *= 2)
        for (int dt = THIN_U8; dt <= THIN_U16; ++dt) {
            std::vector<int> idx;
            for (int k = 0; k < n; ++k) {
                if (cls[k] <= 0 || specs[k].dtype != dt) continue;
                int c = cls[k];
                while (c < spread && specs[k].h / (2 * c) >= 32) c *= 2;
                if (c == C) idx.push_back(k);
            }
            if (!idx.empty()) G->resident.push_back({C, idx});
        }
    // Images too large for a cluster: the wide resident mode (the image held
    // by several clusters of one launch) when at most kWideMax of them are in
    // the call, each then having most of the GPU; the tiled engine otherwise.
    std::vector<int> strips(n, 0), csize(n, 0);
    if (allow_wide && (o.kernel == THIN_KERNEL_AUTO || o.kernel == THIN_KERNEL_RESIDENT)) {
        const size_t limit = resident_smem_limit(16 / G->nw);
        for (int k = 0; k < n; ++k)
            if (cls[k] == 0)
                strips[k] = resident_wide_strips(specs[k].w, specs[k].h, specs[k].dtype, limit, G->nw, &csize[k]);
    }
    int nwide = 0;
    for (int k = 0; k < n; ++k) nwide += cls[k] == 0 && strips[k] > 0;
    const bool use_wide = nwide > 0 && (nwide <= kWideMax || o.kernel == THIN_KERNEL_RESIDENT);
    for (int k = 0; k < n; ++k) {
        if (cls[k] != 0) continue;
        if (use_wide && strips[k] > 0) G->wide.push_back({k, strips[k], csize[k]});
        else G->tiled.push_back(k);
    }
    if (!G->tiled.empty() && o.kernel == THIN_KERNEL_RESIDENT) return THIN_ERR_ARG;  // does not fit on chip
    return THIN_OK;
}

namespace {

// Helper streams of the calling host thread for running launch groups side
// by side (created once per thread and device, kept until the process exits).
struct SideStreams {
    int dev = -1;
    cudaStream_t s[kMaxResidentGroups] = {};
    cudaEvent_t ev[kMaxResidentGroups + 1] = {};
};

cudaError_t side_streams(SideStreams **out)
{
    thread_local SideStreams t;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (t.dev != dev) {
        SideStreams n;
        n.dev = dev;
        for (auto &x : n.s)
            if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking);
        for (auto &x : n.ev)
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
        t = n;
    }
    *out = &t;
    return cudaSuccess;
}

}  // namespace

cudaError_t thread_side_streams(cudaStream_t **side, cudaEvent_t **ev)
{
    SideStreams *ss = nullptr;
    const cudaError_t e = side_streams(&ss);
    if (e != cudaSuccess) return e;
    *side = ss->s;
    *ev = ss->ev;
    return cudaSuccess;
}

int Execution::prepare(const std::vector<JobSpec> &specs_in, const Grouping &G, const thin_options &o,
                       cudaStream_t s, bool async_alloc)
{
    specs = specs_in;
    opt = o;
    async = async_alloc;
    for (const auto &grp : G.resident) {
        std::vector<JobSpec> js;
        for (int k : grp.second) js.push_back(specs[k]);
        res.emplace_back();
        res_idx.push_back(grp.second);
        const int rc =
            resident_prepare(js.data(), int(js.size()), grp.first, G.nw, o, s, async_alloc, &res.back(), 0, done);
        if (rc != THIN_OK) return rc;
    }
    for (const auto &wj : G.wide) {
        wide.emplace_back();
        wide_idx.push_back(wj.job);
        const int rc = resident_prepare(&specs[wj.job], 1, wj.C, G.nw, o, s, async_alloc, &wide.back(), wj.strips);
        if (rc != THIN_OK) return rc;
    }
    if (!G.tiled.empty()) {
        std::vector<JobSpec> js;
        for (int k : G.tiled) js.push_back(specs[k]);
        tiled_idx = G.tiled;
        const int rc = tiled_prepare(js.data(), int(js.size()), o, s, async_alloc, &tiled, tiled_max_grid);
        if (rc != THIN_OK) return rc;
    }
    return THIN_OK;
}

// Resident groups run side by side on helper streams forked from s (a
// group's clusters take SMs as another group's finish); the wide launches and
// the tiled group, whose grid barriers need all their blocks resident at
// once, run after them on s, one after another.
cudaError_t Execution::enqueue(cudaStream_t s, cudaStream_t *side, cudaEvent_t *ev) const
{
    cudaError_t e = cudaSuccess;
    const int ng = int(res.size());
    if (ng == 1) {
        e = resident_enqueue(res[0], s);
    } else if (ng > 1) {
        e = cudaEventRecord(ev[0], s);
        for (int g = 0; g < ng && e == cudaSuccess; ++g) {
            e = cudaStreamWaitEvent(side[g], ev[0], 0);
            if (e == cudaSuccess) e = resident_enqueue(res[g], side[g]);
            if (e == cudaSuccess) e = cudaEventRecord(ev[1 + g], side[g]);
        }
        for (int g = 0; g < ng && e == cudaSuccess; ++g) e = cudaStreamWaitEvent(s, ev[1 + g], 0);
    }
    for (size_t w = 0; w < wide.size() && e == cudaSuccess; ++w) e = resident_enqueue(wide[w], s);
    if (e == cudaSuccess && tiled) e = tiled_enqueue(tiled, s);
    return e;
}

int Execution::collect(cudaStream_t s, thin_stats *out) const
{
    int rc = THIN_OK;
    for (size_t g = 0; g < res.size(); ++g) {
        std::vector<thin_stats> st(res_idx[g].size());
        const int r = resident_collect(res[g], opt, s, st.data());
        for (size_t k = 0; k < st.size(); ++k) out[res_idx[g][k]] = st[k];
        if (r != THIN_OK && (rc == THIN_OK || rc == THIN_ERR_NOT_CONVERGED)) rc = r;
    }
    for (size_t w = 0; w < wide.size(); ++w) {
        thin_stats st;
        const int r = resident_collect(wide[w], opt, s, &st);
        out[wide_idx[w]] = st;
        if (r != THIN_OK && (rc == THIN_OK || rc == THIN_ERR_NOT_CONVERGED)) rc = r;
    }
    if (tiled) {
        std::vector<thin_stats> st(tiled_idx.size());
        const int r = tiled_collect(tiled, opt, s, st.data());
        for (size_t k = 0; k < st.size(); ++k) out[tiled_idx[k]] = st[k];
        if (r != THIN_OK && (rc == THIN_OK || rc == THIN_ERR_NOT_CONVERGED)) rc = r;
    }
    return rc;
}

void Execution::release(cudaStream_t s)
{
    for (auto &r : res) resident_release(r, s);
    res.clear();
    for (auto &r : wide) resident_release(r, s);
    wide.clear();
    if (tiled) tiled_release(tiled, s);
    tiled = nullptr;
}

namespace {

// Runs validated images in one device-driven pass: every launch group
// prepared, enqueued side by side, stats collected if asked for.
int dispatch(const std::vector<JobSpec> &specs, const thin_options &o, cudaStream_t s, thin_stats *out,
             bool allow_wide = true)
{
    if (o.max_phases == 0) {  // nothing may run: every image stays as it is, unconverged
        if (out)
            for (size_t k = 0; k < specs.size(); ++k) {
                std::memset(&out[k], 0, sizeof out[k]);
                out[k].status = THIN_ERR_NOT_CONVERGED;
                out[k].last_change_phase = -1;
                out[k].end_phase = o.start_phase;
            }
        return THIN_ERR_NOT_CONVERGED;
    }
    Grouping G;
    int rc = group_jobs(specs, o, &G, allow_wide);
    if (rc != THIN_OK) return rc;
    SideStreams *ss = nullptr;
    if (G.resident.size() > 1) {
        const cudaError_t e = side_streams(&ss);
        if (e != cudaSuccess) return cuda_status(e);
    }
    Execution X;
    rc = X.prepare(specs, G, o, s, true);
    if (rc == THIN_OK) {
        const cudaError_t e = X.enqueue(s, ss ? ss->s : nullptr, ss ? ss->ev : nullptr);
        if (e != cudaSuccess) rc = cuda_status(e);
        else if (out) rc = X.collect(s, out);
    }
    X.release(s);
    return rc;
}

void noop_stats(const thin_options &o, thin_stats *s)
{
    std::memset(s, 0, sizeof *s);
    s->converged = 1;
    s->last_change_phase = -1;
    s->end_phase = o.start_phase;
}

}  // namespace

}  // namespace thin

using namespace thin;

extern "C" {

void thin_default_options(thin_options *opt)
{
    if (!opt) return;
    std::memset(opt, 0, sizeof *opt);
    opt->rule = THIN_RULE_MAX;
    opt->kernel = THIN_KERNEL_AUTO;
    opt->start_phase = 0;
    opt->max_phases = -1;
}

const char *thin_version(void) { return "gb300-thin 0.1 (sm_103a)"; }

void thin_point_table(uint32_t out[256])
{
    if (!out) return;
    for (int i = 0; i < 256; ++i) out[i] = kPointTable.v[i];
}

void thin_point_table_adj(thin_adj adj, uint32_t out[256])
{
    if (!out) return;
    for (int i = 0; i < 256; ++i) out[i] = adj == THIN_ADJ_4_8 ? kPointTable48.v[i] : kPointTable.v[i];
}

int thin_run(void *img_dev, int w, int h, size_t pitch_bytes, thin_dtype dt, uint32_t lambda, thin_adj adj,
             void *stream, const thin_options *opt, thin_stats *out)
{
    NvtxRange nv("thin_run");
    thin_options o;
    thin_default_options(&o);
    if (opt) o = *opt;
    if (adj != THIN_ADJ_8_4 && adj != THIN_ADJ_4_8) return THIN_ERR_ARG;
    int rc = check_options(o);
    if (rc) return rc;
    rc = check_image(img_dev, w, h, pitch_bytes, dt);
    if (rc < 0) return rc;
    if (rc == 1) {
        if (out) noop_stats(o, out);
        return THIN_OK;
    }
    JobSpec j{img_dev, w, h, pitch_bytes, int(dt), lambda, int(adj)};
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (o.kernel == THIN_KERNEL_NAIVE) return naive_run(j, o, s, out);
    if (o.kernel == THIN_KERNEL_TILED) return tiled_run(&j, 1, o, s, out);
    return dispatch(std::vector<JobSpec>{j}, o, s, out);
}

int thin_batch(const thin_job *jobs, int n, thin_adj adj, void *stream, const thin_options *opt, thin_stats *out)
{
    NvtxRange nv("thin_batch");
    thin_options o;
    thin_default_options(&o);
    if (opt) o = *opt;
    if (n < 0 || (n > 0 && !jobs)) return THIN_ERR_ARG;
    if (adj != THIN_ADJ_8_4 && adj != THIN_ADJ_4_8) return THIN_ERR_ARG;
    int rc = check_options(o);
    if (rc) return rc;
    std::vector<JobSpec> specs;
    std::vector<int> where;
    specs.reserve(n);
    for (int k = 0; k < n; ++k) {
        const thin_job &J = jobs[k];
        const int c = check_image(J.img_dev, J.w, J.h, J.pitch, J.dtype);
        if (c < 0) return c;
        if (c == 1) {
            if (out) noop_stats(o, &out[k]);
            continue;
        }
        specs.push_back(JobSpec{J.img_dev, J.w, J.h, J.pitch, J.dtype, J.lambda, int(adj)});
        where.push_back(k);
    }
    if (specs.empty()) return THIN_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<thin_stats> st(out ? specs.size() : 0);
    if (o.kernel == THIN_KERNEL_NAIVE) {
        rc = THIN_OK;
        for (size_t k = 0; k < specs.size(); ++k) {
            thin_stats tmp;
            const int r = naive_run(specs[k], o, s, &tmp);
            if (out) st[k] = tmp;
            if (r != THIN_OK && rc == THIN_OK) rc = r;
            if (r != THIN_OK && r != THIN_ERR_NOT_CONVERGED) return r;
        }
    } else if (o.kernel == THIN_KERNEL_TILED) {
        rc = tiled_run(specs.data(), int(specs.size()), o, s, out ? st.data() : nullptr);
    } else {
        rc = dispatch(specs, o, s, out ? st.data() : nullptr);
    }
    if (out)
        for (size_t k = 0; k < specs.size(); ++k) out[where[k]] = st[k];
    return rc;
}

}  // extern "C"
