// thin_plan.cu -- batch plans: a fixed set of images prepared once and run
// many times as one CUDA graph.
//
// thin_plan_create does all host work of thin_batch once: argument checks,
// launch groups, the tiled group's autotuned tile shape and halo, device job
// tables, tensor maps, occupancy queries.  It then
// captures the device work of one run -- per-run resets, the resident groups
// forked onto side streams, the tiled group after them -- into a CUDA graph.
// thin_plan_launch is one cudaGraphLaunch.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "thin_internal.h"

struct thin_plan {
    std::vector<thin::JobSpec> specs;   // images that run
    std::vector<int> where;             // specs[k] is the caller's job where[k]
    int n = 0;                          // the caller's job count
    thin_options opt;
    int tile_w = 0, tile_h = 0, halo = 0;  // the tiled group's shape, when autotuned
    bool idle = false;                  // nothing runs (no image with an interior, or max_phases == 0)
    thin::Execution X;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t stream = nullptr;  // the plan's own stream: uploads at create, frees at destroy
    cudaEvent_t done = nullptr;     // recorded after every launch
    bool launched = false;
};

namespace {

void destroy_plan(thin_plan *p)
{
    if (!p) return;
    // no launch of the plan may still use its tables: wait for the last one
    // (launches of one plan do not overlap), not for the rest of the device
    if (p->stream && p->done && p->launched) cudaStreamWaitEvent(p->stream, p->done, 0);
    p->X.release(p->stream);
    if (p->stream) cudaStreamSynchronize(p->stream);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->done) cudaEventDestroy(p->done);
    if (p->stream) cudaStreamDestroy(p->stream);
    delete p;
}

}  // namespace

using namespace thin;

extern "C" {

int thin_plan_create(const thin_job *jobs, int n, thin_adj adj, const thin_options *opt, thin_plan **out)
{
    NvtxRange nv("thin_plan_create");
    if (!out) return THIN_ERR_ARG;
    *out = nullptr;
    thin_options o;
    thin_default_options(&o);
    if (opt) o = *opt;
    if (n < 0 || (n > 0 && !jobs)) return THIN_ERR_ARG;
    if (adj != THIN_ADJ_8_4 && adj != THIN_ADJ_4_8) return THIN_ERR_ARG;
    if (o.rule != THIN_RULE_MAX && o.rule != THIN_RULE_MIN) return THIN_ERR_ARG;
    if (o.op != THIN_OP_THINNING && o.op != THIN_OP_SKELETON) return THIN_ERR_ARG;
    if (o.kernel < THIN_KERNEL_AUTO || o.kernel > THIN_KERNEL_RESIDENT) return THIN_ERR_ARG;
    if (o.kernel == THIN_KERNEL_NAIVE) return THIN_ERR_UNSUPPORTED;  // a host loop per round: nothing to capture
    if (o.start_phase < 0 || o.tile_w < 0 || o.tile_h < 0 || o.halo < 0) return THIN_ERR_ARG;
    thin_plan *p = new thin_plan;
    p->n = n;
    p->opt = o;
    for (int k = 0; k < n; ++k) {
        const thin_job &J = jobs[k];
        if (J.w < 0 || J.h < 0 || (J.dtype != THIN_U8 && J.dtype != THIN_U16)) {
            delete p;
            return THIN_ERR_ARG;
        }
        if (J.w == 0 || J.h == 0) continue;
        const size_t es = elem_size(J.dtype);
        if (!J.img_dev || J.pitch < size_t(J.w) * es ||
            (es == 2 && ((reinterpret_cast<uintptr_t>(J.img_dev) & 1) || (J.pitch & 1)))) {
            delete p;
            return THIN_ERR_ARG;
        }
        if (J.w < 3 || J.h < 3) continue;
        p->specs.push_back(JobSpec{J.img_dev, J.w, J.h, J.pitch, J.dtype, J.lambda, int(adj)});
        p->where.push_back(k);
    }
    p->idle = p->specs.empty() || o.max_phases == 0;
    if (p->idle) {
        *out = p;
        return THIN_OK;
    }
    Grouping G;
    int rc = group_jobs(p->specs, o, &G);
    if (rc != THIN_OK) {
        delete p;
        return rc;
    }
    cudaStream_t cs = nullptr;
    std::vector<cudaStream_t> side(kMaxResidentGroups, nullptr);
    std::vector<cudaEvent_t> ev(kMaxResidentGroups + 1, nullptr);
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    p->stream = cs;
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming);
    for (auto &x : side)
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking);
    for (auto &x : ev)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
    // The tiled group's tile shape and halo depth: autotuned on its largest
    // image (trials on a scratch copy, 64 phases each) unless the caller set them.
    thin_options ot = o;
    if (e == cudaSuccess && !G.tiled.empty() && o.tile_w == 0 && o.tile_h == 0 && o.halo == 0) {
        int big = G.tiled[0];
        for (int k : G.tiled)
            if (double(p->specs[k].w) * p->specs[k].h > double(p->specs[big].w) * p->specs[big].h) big = k;
        const JobSpec &J = p->specs[big];
        thin_options tuned = o;
        if (thin_autotune(J.img, J.w, J.h, J.pitch, thin_dtype(J.dtype), J.lam, cs, 64, &tuned, nullptr) == THIN_OK) {
            // a u16 image in the group caps the halo at 8; autotune tried that image's dtype only
            bool any16 = false;
            for (int k : G.tiled) any16 |= p->specs[k].dtype == THIN_U16;
            if (!any16 || tuned.halo <= 8) ot = tuned;
        }
        p->tile_w = ot.tile_w;
        p->tile_h = ot.tile_h;
        p->halo = ot.halo;
    }
    if (e == cudaSuccess) {
        rc = p->X.prepare(p->specs, G, ot, cs, true);  // plan-owned device memory, stream-ordered on cs
        if (rc == THIN_OK) e = cudaStreamSynchronize(cs);  // tables uploaded before capture
        if (rc == THIN_OK && e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (rc == THIN_OK && e == cudaSuccess) {
            const cudaError_t ee = p->X.enqueue(cs, side.data(), ev.data());
            e = cudaStreamEndCapture(cs, &p->graph);
            if (ee != cudaSuccess) e = ee;
        }
        if (rc == THIN_OK && e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    }
    for (auto x : ev)
        if (x) cudaEventDestroy(x);
    for (auto x : side)
        if (x) cudaStreamDestroy(x);
    if (rc == THIN_OK && e != cudaSuccess) rc = cuda_status(e);
    if (rc != THIN_OK) {
        destroy_plan(p);
        return rc;
    }
    *out = p;
    return THIN_OK;
}

int thin_plan_launch(thin_plan *p, void *stream)
{
    NvtxRange nv("thin_plan_launch");
    if (!p) return THIN_ERR_ARG;
    if (p->idle) return THIN_OK;
    cudaError_t e = cudaGraphLaunch(p->exec, static_cast<cudaStream_t>(stream));
    if (e == cudaSuccess) e = cudaEventRecord(p->done, static_cast<cudaStream_t>(stream));
    if (e == cudaSuccess) p->launched = true;
    return cuda_status(e);
}

int thin_plan_stats(thin_plan *p, void *stream, thin_stats *out)
{
    if (!p || (!out && p->n > 0)) return THIN_ERR_ARG;
    const thin_options &o = p->opt;
    for (int k = 0; k < p->n; ++k) {  // images that do not run: finished as they are
        std::memset(&out[k], 0, sizeof out[k]);
        out[k].converged = 1;
        out[k].last_change_phase = -1;
        out[k].end_phase = o.start_phase;
    }
    if (p->specs.empty()) return THIN_OK;
    if (o.max_phases == 0) {
        for (int k : p->where) {
            out[k].converged = 0;
            out[k].status = THIN_ERR_NOT_CONVERGED;
        }
        return THIN_ERR_NOT_CONVERGED;
    }
    std::vector<thin_stats> st(p->specs.size());
    const int rc = p->X.collect(static_cast<cudaStream_t>(stream), st.data());
    for (size_t k = 0; k < st.size(); ++k) out[p->where[k]] = st[k];
    return rc;
}

int thin_plan_tiling(const thin_plan *p, int *tile_w, int *tile_h, int *halo)
{
    if (!p || !tile_w || !tile_h || !halo) return THIN_ERR_ARG;
    *tile_w = p->tile_w;
    *tile_h = p->tile_h;
    *halo = p->halo;
    return THIN_OK;
}

int thin_plan_destroy(thin_plan *p)
{
    if (!p) return THIN_ERR_ARG;
    destroy_plan(p);
    return THIN_OK;
}

}  // extern "C"
