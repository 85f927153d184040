// C-ABI glue: thread-local error messages, status names, deferred checks.
#include <stdarg.h>
#include <stdio.h>

#include "aica_internal.cuh"

namespace aica {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

aica_status cuda_fail(cudaError_t e, const char *what) {
    set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
    return e == cudaErrorMemoryAllocation ? AICA_ERR_OOM : AICA_ERR_CUDA;
}

}  // namespace aica

extern "C" const char *aica_last_error(void) { return aica::g_err; }

extern "C" const char *aica_status_string(aica_status s) {
    switch (s) {
        case AICA_OK: return "AICA_OK";
        case AICA_ERR_INVALID_ARG: return "AICA_ERR_INVALID_ARG";
        case AICA_ERR_BAD_MESH: return "AICA_ERR_BAD_MESH";
        case AICA_ERR_OUTSIDE_MESH: return "AICA_ERR_OUTSIDE_MESH";
        case AICA_ERR_NOT_BUILT: return "AICA_ERR_NOT_BUILT";
        case AICA_ERR_CAPACITY: return "AICA_ERR_CAPACITY";
        case AICA_ERR_CUDA: return "AICA_ERR_CUDA";
        case AICA_ERR_OOM: return "AICA_ERR_OOM";
    }
    return "AICA_UNKNOWN_STATUS";
}

extern "C" aica_status aica_set_deferred_checks(aica_mesh *m, int deferred) {
    if (!m) { aica::set_error("aica_set_deferred_checks: mesh is NULL"); return AICA_ERR_INVALID_ARG; }
    m->deferred = deferred != 0;
    return AICA_OK;
}

extern "C" aica_status aica_check_status(aica_mesh *m, void *stream) {
    if (!m) { aica::set_error("aica_check_status: mesh is NULL"); return AICA_ERR_INVALID_ARG; }
    unsigned flags[2] = {0, 0};
    cudaStream_t st = (cudaStream_t)stream;
    AICA_CUDA(cudaMemcpyAsync(flags, m->flags.p, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    AICA_CUDA(cudaStreamSynchronize(st));
    AICA_CUDA(cudaGetLastError());
    // reported once: the error bits start again from zero
    if (flags[0]) AICA_CUDA(cudaMemsetAsync(m->flags.p, 0, sizeof(unsigned), st));
    if (flags[0] & aica::kFlagSpecies) { aica::set_error("species index out of range"); return AICA_ERR_INVALID_ARG; }
    if (flags[0] & aica::kFlagOutside) { aica::set_error("some molecules lie in no cell"); return AICA_ERR_OUTSIDE_MESH; }
    if (flags[0] & aica::kFlagCapacity) { aica::set_error("a kernel capacity was exceeded"); return AICA_ERR_CAPACITY; }
    if (flags[0] & aica::kFlagTimeout) { aica::set_error("a bounded wait between blocks timed out"); return AICA_ERR_CUDA; }
    return AICA_OK;
}

extern "C" aica_status aica_get_work_counters(aica_mesh *m, int64_t *out, void *stream) {
    if (!m || !out) { aica::set_error("aica_get_work_counters: NULL argument"); return AICA_ERR_INVALID_ARG; }
    if (!m->acc.p) { out[0] = out[1] = 0; return AICA_OK; }
    unsigned long long v[2];
    cudaStream_t st = (cudaStream_t)stream;
    AICA_CUDA(cudaMemcpyAsync(v, (const unsigned long long *)m->acc.p + 14, sizeof(v), cudaMemcpyDeviceToHost, st));
    AICA_CUDA(cudaStreamSynchronize(st));
    out[0] = (int64_t)v[0];
    out[1] = (int64_t)v[1];
    return AICA_OK;
}

extern "C" aica_status aica_set_option(aica_mesh *m, aica_option opt, double v) {
    if (!m) { aica::set_error("aica_set_option: mesh is NULL"); return AICA_ERR_INVALID_ARG; }
    switch (opt) {
    case AICA_OPT_FP32_REFINE_TOL: m->refine_tol = v; return AICA_OK;
    case AICA_OPT_COUNT_EVALUATED: m->count_evaluated = v != 0; return AICA_OK;
    case AICA_OPT_FP32_KERNEL:
        if (v != 0 && v != 1) break;
        m->fp32_kernel = (int)v;
        return AICA_OK;
    case AICA_OPT_N_OWNED:
        if (!(v >= -1) || v != (double)(int64_t)v) break;
        m->n_owned = (int64_t)v;
        return AICA_OK;
    default: break;
    }
    aica::set_error("aica_set_option: unknown, read-only or invalid option %d = %g", (int)opt, v);
    return AICA_ERR_INVALID_ARG;
}

extern "C" aica_status aica_get_option(aica_mesh *m, aica_option opt, double *v, void *stream) {
    if (!m || !v) { aica::set_error("aica_get_option: NULL argument"); return AICA_ERR_INVALID_ARG; }
    switch (opt) {
    case AICA_OPT_FP32_REFINE_TOL: *v = m->refine_tol; return AICA_OK;
    case AICA_OPT_COUNT_EVALUATED: *v = m->count_evaluated ? 1 : 0; return AICA_OK;
    case AICA_OPT_FP32_KERNEL: *v = m->fp32_kernel; return AICA_OK;
    case AICA_OPT_CLUSTER_PATH: *v = m->built && m->n_cl_runs >= 0 ? 1 : 0; return AICA_OK;
    case AICA_OPT_N_OWNED: *v = (double)m->n_owned; return AICA_OK;
    case AICA_OPT_REFINED: {
        int n = 0;
        if (m->flag_list.p) {
            cudaStream_t st = (cudaStream_t)stream;
            AICA_CUDA(cudaMemcpyAsync(&n, m->flag_list.p, sizeof(int), cudaMemcpyDeviceToHost, st));
            AICA_CUDA(cudaStreamSynchronize(st));
        }
        *v = n;
        return AICA_OK;
    }
    default: break;
    }
    aica::set_error("aica_get_option: unknown option %d", (int)opt);
    return AICA_ERR_INVALID_ARG;
}

extern "C" int64_t aica_last_launch_count(const aica_mesh *m) { return m ? m->launches : 0; }

extern "C" aica_status aica_set_kernel_timing(aica_mesh *m, int enable) {
    if (!m) { aica::set_error("aica_set_kernel_timing: mesh is NULL"); return AICA_ERR_INVALID_ARG; }
    m->timing = enable != 0;
    return AICA_OK;
}

extern "C" aica_status aica_take_kernel_times(aica_mesh *m, float *ms, int64_t cap, int64_t *n) {
    if (!m || !n || (cap > 0 && !ms)) { aica::set_error("aica_take_kernel_times: NULL argument"); return AICA_ERR_INVALID_ARG; }
    int64_t k = 0;
    for (auto &p : m->tev) {
        AICA_CUDA(cudaEventSynchronize(p.second));
        float t = 0;
        AICA_CUDA(cudaEventElapsedTime(&t, p.first, p.second));
        if (k < cap) ms[k] = t;
        ++k;
        m->tfree.push_back(p);
    }
    m->tev.clear();
    *n = k < cap ? k : cap;
    return AICA_OK;
}

namespace aica {
// start/stop events around a measured kernel (see aica_set_kernel_timing)
cudaError_t timing_begin(aica_mesh *m, cudaStream_t st, cudaEvent_t *stop) {
    *stop = nullptr;
    if (!m->timing) return cudaSuccess;
    std::pair<cudaEvent_t, cudaEvent_t> p;
    if (!m->tfree.empty()) {
        p = m->tfree.back();
        m->tfree.pop_back();
    } else {
        cudaError_t e = cudaEventCreate(&p.first);
        if (e == cudaSuccess) e = cudaEventCreate(&p.second);
        if (e != cudaSuccess) return e;
    }
    m->tev.push_back(p);
    *stop = p.second;
    return cudaEventRecord(p.first, st);
}
cudaError_t timing_end(cudaEvent_t stop, cudaStream_t st) { return stop ? cudaEventRecord(stop, st) : cudaSuccess; }
}  // namespace aica
