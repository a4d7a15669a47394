/* An NVTX tool for tests/test_nvtx.py (test infrastructure only): loaded by
 * the NVTX v3 headers through NVTX_INJECTION64_PATH, it takes over the
 * domain-creation and range push / pop entry points and writes one line per
 * range event of the domain "libsmc" to the file named by
 * SMC_NVTX_PROBE_OUT. */
#define NVTX_NO_IMPL
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

static nvtxDomainHandle_t smc_domain = NULL;
static FILE* out = NULL;
static int depth = 0;

static nvtxDomainHandle_t NVTX_API probe_domain_create(const char* name) {
  static intptr_t next = 1;
  nvtxDomainHandle_t h = (nvtxDomainHandle_t)(next++);
  if (name && strcmp(name, "libsmc") == 0) smc_domain = h;
  return h;
}

static int NVTX_API probe_push(nvtxDomainHandle_t d, const nvtxEventAttributes_t* a) {
  if (d == smc_domain && a && a->messageType == NVTX_MESSAGE_TYPE_ASCII) fprintf(out, "push %s\n", a->message.ascii);
  return depth++;
}

static int NVTX_API probe_pop(nvtxDomainHandle_t d) {
  if (d == smc_domain) fprintf(out, "pop\n");
  return --depth;
}

int InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get_table) {
  const NvtxExportTableCallbacks* cb = (const NvtxExportTableCallbacks*)get_table(NVTX_ETID_CALLBACKS);
  NvtxFunctionTable table = NULL;
  unsigned int size = 0;
  if (!cb || !cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE2, &table, &size)) return 0;
  if (size <= NVTX_CBID_CORE2_DomainCreateA) return 0;
  const char* path = getenv("SMC_NVTX_PROBE_OUT");
  out = path ? fopen(path, "w") : stderr;
  if (!out) return 0;
  setvbuf(out, NULL, _IOLBF, 0);
  *table[NVTX_CBID_CORE2_DomainCreateA] = (NvtxFunctionPointer)probe_domain_create;
  *table[NVTX_CBID_CORE2_DomainRangePushEx] = (NvtxFunctionPointer)probe_push;
  *table[NVTX_CBID_CORE2_DomainRangePop] = (NvtxFunctionPointer)probe_pop;
  return 1;
}
