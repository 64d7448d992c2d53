// Runtime support of the library: logging, device allocation with host-side
// fault injection and scratch poisoning, and NVTX ranges.
//
// Environment (read when used, so a process can change them between calls):
//   WD_LOG=<level>            log to stderr: 0 off (default), 1 errors, 2 warnings,
//                             3 info (contexts, rules, servers), 4 debug (allocations)
//   WD_FAULT_ALLOC=<n>        the n-th device allocation after the variable takes
//                             this value fails with WD_ENOMEM (host-side; no GPU fault)
//   WD_FAULT_DROP_COMPLETION=<n>
//                             a server started while it is set never delivers its
//                             n-th completion, so the client's wait runs out (WD_ETIMEOUT)
//   WD_POISON_SCRATCH=1       fill every device allocation with 0xFF bytes (NaN as
//                             float64 and float32) before use, so a read of memory the
//                             library did not write shows up as NaN in the results
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <string>

#include "wd_internal.h"

namespace {

int env_int(const char* name, int dflt)
{
    const char* v = std::getenv(name);
    if (!v || !*v) return dflt;
    char* end = nullptr;
    const long x = std::strtol(v, &end, 10);
    return (end && *end == '\0') ? (int)x : dflt;
}

std::mutex g_alloc_mu;
std::string g_fault_val;  // value of WD_FAULT_ALLOC the counter belongs to
int64_t g_fault_count = 0;

}  // namespace

int wd_log_level() { return env_int("WD_LOG", 0); }

void wd_log(int level, const char* fmt, ...)
{
    if (level > wd_log_level()) return;
    static const char* names[] = {"", "error", "warn", "info", "debug"};
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    std::fprintf(stderr, "[wd %s] %s\n", names[level < 1 ? 1 : (level > 4 ? 4 : level)], buf);
}

bool wd_fault_alloc_now()
{
    const char* v = std::getenv("WD_FAULT_ALLOC");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    const std::string cur = v ? v : "";
    if (cur != g_fault_val) {
        g_fault_val = cur;
        g_fault_count = 0;
    }
    if (cur.empty()) return false;
    const int n = env_int("WD_FAULT_ALLOC", 0);
    if (n <= 0) return false;
    return ++g_fault_count == n;
}

int wd_fault_drop_completion() { return env_int("WD_FAULT_DROP_COMPLETION", 0); }

cudaError_t wd_dev_alloc(void** p, size_t bytes, const char* what)
{
    *p = nullptr;
    if (wd_fault_alloc_now()) {
        wd_log(2, "injected allocation failure: %s (%zu bytes)", what, bytes);
        return cudaErrorMemoryAllocation;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        wd_log(1, "cudaMalloc failed: %s (%zu bytes): %s", what, bytes, cudaGetErrorString(e));
        return e;
    }
    wd_log(4, "alloc %s: %zu bytes", what, bytes);
    if (env_int("WD_POISON_SCRATCH", 0) != 0 && bytes > 0) e = cudaMemset(*p, 0xFF, bytes);
    return e;
}

#include <nvtx3/nvToolsExt.h>

WdRange::WdRange(const char* name) { nvtxRangePushA(name); }
WdRange::~WdRange() { nvtxRangePop(); }
