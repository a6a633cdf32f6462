/* NVTX injection library for the tests: named by NVTX_INJECTION64_PATH, it
 * is loaded by the first NVTX call of the process and records every range
 * push (with its message) and pop in the file named by EWALD_NVTX_LOG, one
 * line each.  Test infrastructure only. */
#include <stdio.h>
#include <stdlib.h>

#include <nvtx3/nvToolsExt.h>

static FILE *g_log;

static int record_push(const char *message) {
    if (g_log) {
        fprintf(g_log, "push %s\n", message ? message : "");
        fflush(g_log);
    }
    return 0;
}

static int record_pop(void) {
    if (g_log) {
        fprintf(g_log, "pop\n");
        fflush(g_log);
    }
    return 0;
}

int InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get_table) {
    const NvtxExportTableCallbacks *cb = (const NvtxExportTableCallbacks *)get_table(NVTX_ETID_CALLBACKS);
    NvtxFunctionTable table = 0;
    unsigned int size = 0;
    const char *path = getenv("EWALD_NVTX_LOG");
    if (!cb || !path) return 0;
    cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE, &table, &size);
    if (!table || size <= NVTX_CBID_CORE_RangePop) return 0;
    *table[NVTX_CBID_CORE_RangePushA] = (NvtxFunctionPointer)record_push;
    *table[NVTX_CBID_CORE_RangePop] = (NvtxFunctionPointer)record_pop;
    g_log = fopen(path, "w");
    return g_log != 0;
}
