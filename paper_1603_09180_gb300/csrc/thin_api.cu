// thin_api.cu -- the C-ABI of libthin.so: argument checks and dispatch.
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

namespace {

int check_options(const thin_options &o)
{
    if (o.rule != THIN_RULE_MAX && o.rule != THIN_RULE_MIN) return THIN_ERR_ARG;
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

// Runs images on the resident engine where they fit (AUTO, RESIDENT) and on
// the tiled engine otherwise; stats land at the images' own positions.
int dispatch(const std::vector<JobSpec> &specs, const thin_options &o, cudaStream_t s, thin_stats *out)
{
    const int n = int(specs.size());
    const int nw = 16;  // warps per resident block (one block per SM measured fastest)
    std::vector<int> cls(n, 0);
    if (o.kernel == THIN_KERNEL_AUTO || o.kernel == THIN_KERNEL_RESIDENT) {
        const size_t limit = resident_smem_limit(16 / nw);
        for (int k = 0; k < n; ++k)
            cls[k] = resident_cluster_size(specs[k].w, specs[k].h, specs[k].dtype, limit, nw, nullptr, nullptr);
    }
    int eligible = 0, sms = 0, dev = 0;
    for (int k = 0; k < n; ++k) eligible += cls[k] > 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // few images: spread each over more blocks of a wider cluster
    int spread = 1;
    while (eligible > 0 && spread < 8 && spread * 2 * eligible <= sms * (16 / nw)) spread *= 2;
    int rc = THIN_OK;
    for (int C = 1; C <= 8; C *= 2) {
        std::vector<JobSpec> group;
        std::vector<int> where;
        for (int k = 0; k < n; ++k) {
            if (cls[k] <= 0) continue;
            int c = cls[k];  // spread, but keep at least 32 rows per block
            while (c < spread && specs[k].h / (2 * c) >= 32) c *= 2;
            if (c == C) {
                group.push_back(specs[k]);
                where.push_back(k);
            }
        }
        if (group.empty()) continue;
        std::vector<thin_stats> st(out ? group.size() : 0);
        const int r = resident_run(group.data(), int(group.size()), C, nw, o, s, out ? st.data() : nullptr);
        if (out)
            for (size_t k = 0; k < group.size(); ++k) out[where[k]] = st[k];
        if (r != THIN_OK && r != THIN_ERR_NOT_CONVERGED) return r;
        if (r != THIN_OK && rc == THIN_OK) rc = r;
    }
    std::vector<JobSpec> rest;
    std::vector<int> where;
    for (int k = 0; k < n; ++k)
        if (cls[k] == 0) {
            rest.push_back(specs[k]);
            where.push_back(k);
        }
    if (!rest.empty()) {
        if (o.kernel == THIN_KERNEL_RESIDENT) return THIN_ERR_ARG;  // does not fit on chip
        std::vector<thin_stats> st(out ? rest.size() : 0);
        const int r = tiled_run(rest.data(), int(rest.size()), o, s, out ? st.data() : nullptr);
        if (out)
            for (size_t k = 0; k < rest.size(); ++k) out[where[k]] = st[k];
        if (r != THIN_OK && r != THIN_ERR_NOT_CONVERGED) return r;
        if (r != THIN_OK && rc == THIN_OK) rc = r;
    }
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

int thin_run(void *img_dev, int w, int h, size_t pitch_bytes, thin_dtype dt, uint32_t lambda, thin_adj adj,
             void *stream, const thin_options *opt, thin_stats *out)
{
    thin_options o;
    thin_default_options(&o);
    if (opt) o = *opt;
    if (adj == THIN_ADJ_4_8) return THIN_ERR_UNSUPPORTED;
    if (adj != THIN_ADJ_8_4) return THIN_ERR_ARG;
    int rc = check_options(o);
    if (rc) return rc;
    rc = check_image(img_dev, w, h, pitch_bytes, dt);
    if (rc < 0) return rc;
    if (rc == 1) {
        if (out) noop_stats(o, out);
        return THIN_OK;
    }
    JobSpec j{img_dev, w, h, pitch_bytes, int(dt), lambda};
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (o.kernel == THIN_KERNEL_NAIVE) return naive_run(j, o, s, out);
    if (o.kernel == THIN_KERNEL_TILED) return tiled_run(&j, 1, o, s, out);
    return dispatch(std::vector<JobSpec>{j}, o, s, out);
}

int thin_batch(const thin_job *jobs, int n, thin_adj adj, void *stream, const thin_options *opt, thin_stats *out)
{
    thin_options o;
    thin_default_options(&o);
    if (opt) o = *opt;
    if (n < 0 || (n > 0 && !jobs)) return THIN_ERR_ARG;
    if (adj == THIN_ADJ_4_8) return THIN_ERR_UNSUPPORTED;
    if (adj != THIN_ADJ_8_4) return THIN_ERR_ARG;
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
        specs.push_back(JobSpec{J.img_dev, J.w, J.h, J.pitch, J.dtype, J.lambda});
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
