/* NVTX tool for the tracing test: a shared library that the NVTX 3 headers
 * load when NVTX_INJECTION64_PATH names it (the documented tool hook), taking
 * over nvtxRangePushA / nvtxRangePop and appending one line per call to the
 * file named by DSPS_NVTX_LOG.  Test infrastructure only. */
#include <stdio.h>
#include <stdlib.h>

#include <nvtx3/nvToolsExt.h>

static FILE *g_log;

static int range_push_a(const char *message) {
    if (g_log) {
        fprintf(g_log, "push %s\n", message ? message : "");
        fflush(g_log);
    }
    return 0;
}

static int range_pop(void) {
    if (g_log) {
        fprintf(g_log, "pop\n");
        fflush(g_log);
    }
    return 0;
}

int InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get_export_table) {
    const char *path = getenv("DSPS_NVTX_LOG");
    g_log = path ? fopen(path, "a") : NULL;
    const NvtxExportTableCallbacks *cb =
        (const NvtxExportTableCallbacks *)get_export_table(NVTX_ETID_CALLBACKS);
    if (!cb) return 0;
    NvtxFunctionTable table = 0;
    unsigned int size = 0;
    if (!cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE, &table, &size) || !table) return 0;
    *table[NVTX_CBID_CORE_RangePushA] = (NvtxFunctionPointer)range_push_a;
    *table[NVTX_CBID_CORE_RangePop] = (NvtxFunctionPointer)range_pop;
    return 1;
}
