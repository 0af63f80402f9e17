/* NVTX injection library for the tests (test infrastructure): when a process names it in
 * NVTX_INJECTION64_PATH, the NVTX calls of that process land here. It records the domains
 * created and the ranges pushed and popped, which the test reads through nvtx_probe_*.
 * Uses only the NVTX v3 tool interface declared in the CUDA toolkit's nvtx3 headers. */
#include <stdint.h>
#include <string.h>

#include <nvtx3/nvToolsExt.h>

#define MAX_NAMES 4096
static char g_names[MAX_NAMES][64];
static int g_n_push = 0, g_n_pop = 0, g_depth = 0, g_max_depth = 0;
static char g_domain[64];
static int g_domain_handle = 1;

static nvtxDomainHandle_t probe_domain_create(const char *name)
{
    strncpy(g_domain, name ? name : "", sizeof g_domain - 1);
    return (nvtxDomainHandle_t)&g_domain_handle;
}

static int probe_push(nvtxDomainHandle_t d, const nvtxEventAttributes_t *a)
{
    (void)d;
    if (g_n_push < MAX_NAMES) {
        const char *m = a && a->messageType == NVTX_MESSAGE_TYPE_ASCII && a->message.ascii ? a->message.ascii : "";
        strncpy(g_names[g_n_push], m, 63);
    }
    g_n_push++;
    g_depth++;
    if (g_depth > g_max_depth) g_max_depth = g_depth;
    return g_depth - 1;
}

static int probe_pop(nvtxDomainHandle_t d)
{
    (void)d;
    g_n_pop++;
    g_depth--;
    return g_depth;
}

int InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get)
{
    const NvtxExportTableCallbacks *cb = (const NvtxExportTableCallbacks *)get(NVTX_ETID_CALLBACKS);
    NvtxFunctionTable table = 0;
    unsigned int size = 0;
    if (!cb || !cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE2, &table, &size) || !table) return 0;
    if (size <= NVTX_CBID_CORE2_DomainCreateA) return 0;
    *table[NVTX_CBID_CORE2_DomainCreateA] = (NvtxFunctionPointer)probe_domain_create;
    *table[NVTX_CBID_CORE2_DomainRangePushEx] = (NvtxFunctionPointer)probe_push;
    *table[NVTX_CBID_CORE2_DomainRangePop] = (NvtxFunctionPointer)probe_pop;
    return 1;
}

/* read-out for the test */
int nvtx_probe_pushes(void) { return g_n_push; }
int nvtx_probe_pops(void) { return g_n_pop; }
int nvtx_probe_max_depth(void) { return g_max_depth; }
const char *nvtx_probe_name(int i) { return i >= 0 && i < g_n_push && i < MAX_NAMES ? g_names[i] : ""; }
const char *nvtx_probe_domain(void) { return g_domain; }
