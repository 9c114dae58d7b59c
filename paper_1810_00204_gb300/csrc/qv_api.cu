// qv_api.cu -- error reporting and device queries shared by the entry points.
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include <nvtx3/nvToolsExt.h>

#include "qv_common.cuh"

namespace {
thread_local char g_last_error[512] = "";
}

qv_status qv_set_error(qv_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return st;
}

qv_status qv_check_cuda(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return QV_OK;
    return qv_set_error(QV_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

unsigned qv_cross_spin_limit() {
    const char *f = std::getenv("QVTS_FAULT");
    return (f && std::strcmp(f, "timeout") == 0) ? 0u : qv::kSpinLimit;
}

qv_status qv_injected_fault(const char *where, bool takes_workspace) {
    const char *f = std::getenv("QVTS_FAULT");
    if (!f) return QV_OK;
    if (takes_workspace && std::strcmp(f, "oom") == 0)
        return qv_set_error(QV_ERR_WORKSPACE, "%s: injected fault (QVTS_FAULT=oom): the workspace cannot hold the call",
                            where);
    if (std::strcmp(f, "invalid") == 0)
        return qv_set_error(QV_ERR_INVALID, "%s: injected fault (QVTS_FAULT=invalid)", where);
    return QV_OK;
}

unsigned qv_bounds_injected_site() {
    const char *f = std::getenv("QVTS_FAULT");
    return (f && std::strcmp(f, "bounds") == 0) ? 1u : 0u;
}

QvRange::QvRange(const char *name) {
    char b[96];
    std::snprintf(b, sizeof(b), "qvts:%s", name);
    nvtxRangePushA(b);
}

QvRange::QvRange(const char *name, int level) {
    char b[96];
    std::snprintf(b, sizeof(b), "qvts:%s level %d", name, level);
    nvtxRangePushA(b);
}

QvRange::~QvRange() { nvtxRangePop(); }

int qv_num_sms() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

extern "C" const char *qv_last_error(void) { return g_last_error; }

extern "C" const char *qv_version(void) { return "qvts-gb300 0.1 (sm_103a)"; }
