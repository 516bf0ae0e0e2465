// dl_debug.cu -- host-side fault injection for the library's allocations, and NVTX ranges.
//
// DL_FAULT (environment, read at every allocation, so a process may change it between calls):
//   alloc@k    the k-th allocation made after DL_FAULT took this value fails, once
//   alloc@k+   the k-th allocation and every one after it fail
// "Allocation" is every device buffer and pinned host buffer the library asks CUDA for
// (workspace growth, program relations, serving slot set-up).  A failed allocation is reported
// to the caller as DL_ENOMEM with the usual message; nothing on the GPU is made to fail.  Any
// other value is ignored with one warning on stderr.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>

#include "dl_internal.h"

namespace dl {

namespace {

struct FaultPlan {
    std::mutex mu;
    std::string spec;   // the value the counter belongs to
    long long at = 0;   // 0: no fault
    bool sticky = false;
    long long count = 0;
    bool warned = false;
};

FaultPlan &plan() {
    static FaultPlan p;
    return p;
}

// Whether the next allocation must fail (and count it).
bool next_alloc_fails() {
    const char *env = std::getenv("DL_FAULT");
    FaultPlan &p = plan();
    std::lock_guard<std::mutex> lk(p.mu);
    const std::string cur = env ? env : "";
    if (cur != p.spec) {  // a new plan: parse it and restart the count
        p.spec = cur;
        p.at = 0;
        p.sticky = false;
        p.count = 0;
        if (!cur.empty()) {
            long long k = 0;
            char tail[4] = {0};
            const int got = std::sscanf(cur.c_str(), "alloc@%lld%3s", &k, tail);
            if (got >= 1 && k >= 1 && (got == 1 || std::strcmp(tail, "+") == 0)) {
                p.at = k;
                p.sticky = got == 2;
            } else if (!p.warned) {
                std::fprintf(stderr, "libdl: DL_FAULT=\"%s\" not understood (alloc@k or alloc@k+); ignored\n",
                             cur.c_str());
                p.warned = true;
            }
        }
    }
    if (p.at == 0) return false;
    ++p.count;
    return p.sticky ? p.count >= p.at : p.count == p.at;
}

}  // namespace

cudaError_t device_alloc(void **ptr, size_t bytes) {
    if (next_alloc_fails()) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(ptr, bytes);
}

cudaError_t host_pinned_alloc(void **ptr, size_t bytes) {
    if (next_alloc_fails()) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocHost(ptr, bytes);
}

}  // namespace dl
