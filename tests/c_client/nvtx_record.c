/*
 * nvtx_record.c -- a minimal NVTX v3 tool for the tests: loaded through
 * NVTX_INJECTION64_PATH, it takes over nvtxRangePushA / nvtxRangePop and
 * appends one line per event to the file named by QVTS_NVTX_LOG
 * ("push <name>" or "pop").  It lets a CPU-only test see which ranges the
 * library opens and that every one is closed.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <nvtx3/nvToolsExt.h>

static FILE *g_log;

static int rec_push(const char *msg) {
    if (g_log) {
        fprintf(g_log, "push %s\n", msg ? msg : "");
        fflush(g_log);
    }
    return 0;
}

static int rec_pop(void) {
    if (g_log) {
        fputs("pop\n", g_log);
        fflush(g_log);
    }
    return 0;
}

int InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get_table) {
    const char *path = getenv("QVTS_NVTX_LOG");
    if (!path || !get_table) return 0;
    g_log = fopen(path, "a");
    if (!g_log) return 0;
    const NvtxExportTableCallbacks *cb = (const NvtxExportTableCallbacks *)get_table(NVTX_ETID_CALLBACKS);
    if (!cb || !cb->GetModuleFunctionTable) return 0;
    NvtxFunctionTable table = 0;
    unsigned int size = 0;
    if (!cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE, &table, &size) || !table) return 0;
    if (size <= NVTX_CBID_CORE_RangePop) return 0;
    *table[NVTX_CBID_CORE_RangePushA] = (NvtxFunctionPointer)rec_push;
    *table[NVTX_CBID_CORE_RangePop] = (NvtxFunctionPointer)rec_pop;
    return 1;
}
