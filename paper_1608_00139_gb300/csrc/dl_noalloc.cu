// dl_noalloc.cu -- transitive closure for callers that cannot allocate device memory.
//
// dl_tc_closure() keeps its working matrices in buffers that its context allocates with
// cudaMalloc.  Some callers cannot let a library do that: a process whose device memory is
// entirely reserved by another framework's pool, a latency-critical loop where cudaMalloc's
// implicit device synchronisation is not acceptable, or a plug-in that must not touch the
// allocator of its host application.  This file gives them one entry point,
// dl_tc_closure_noalloc(), that computes the same model with the same kernels but keeps all
// of its scratch in one fixed-size array compiled into the library (g_noalloc_scratch below).
//
// Costs and rules of that array:
//   - every GPU that loads libdl holds kNoallocBytes (about 9 MiB) for it until the process
//     exits, whether or not the entry point is ever called;
//   - it bounds the problem size: n <= DL_NOALLOC_MAX_N (2048);
//   - every call on a device shares it, and it keeps the previous call's contents; each call
//     clears or fully rewrites what it reads, so results never depend on an earlier call;
//   - two calls whose work overlaps on the GPU (different streams or host threads) race on
//     it and give wrong results: serialise them.
// The host cannot use the array's name as a device address.  Every call asks the runtime for
// the address with cudaGetSymbolAddress (with the caller's device current); nothing is cached,
// so a context that was destroyed and re-created (cudaDeviceReset) never leaves a stale
// pointer behind.
//
// Module loading: CUDA loads a library's device code lazily by default (CUDA_MODULE_LOADING
// unset or LAZY), so the array and the kernels this entry point launches are placed on a device
// the first time they are needed there, and that first placement is a driver allocation.  A
// caller that reserves the device's memory for its own pool makes one call with n = 0 on each
// device first (before the reservation): it looks up the array and loads every kernel the entry
// point uses, and allocates nothing afterwards.  With CUDA_MODULE_LOADING=EAGER the driver does
// all of that when the library is loaded.
//
// The call is synchronous (it waits on its stream and copies small counters to pageable host
// memory), so it cannot be made while `stream`, or the legacy stream under global capture mode,
// is being captured into a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "../../include/dl.h"
#include "dl_ctx.h"
#include "dl_internal.h"

namespace dl {
namespace {

constexpr int64_t kMaxN = DL_NOALLOC_MAX_N;           // largest n accepted
constexpr int64_t kMaxNp = kMaxN;                     // padded size (kMaxN is a multiple of 256)
constexpr int64_t kMatBytes = kMaxNp * kMaxNp;        // one e4m3 operand
constexpr int64_t kBitsBytes = kMaxNp * (kMaxNp / 64) * 8;
constexpr int64_t kTableBytes = 4096;                 // two GEMM problem descriptors
constexpr int64_t kScalarBytes = 4096;                // counters and the status word
constexpr int64_t kOffC0 = 0;
constexpr int64_t kOffC1 = kOffC0 + kMatBytes;
constexpr int64_t kOffRBits = kOffC1 + kMatBytes;
constexpr int64_t kOffMBits = kOffRBits + kBitsBytes;
constexpr int64_t kOffTable = kOffMBits + kBitsBytes;
constexpr int64_t kOffScalars = kOffTable + kTableBytes;
constexpr int64_t kNoallocBytes = kOffScalars + kScalarBytes;

static_assert(kMaxN % 256 == 0, "the bound must be a multiple of the GEMM tile size");
static_assert(2 * sizeof(GemmProblem) <= kTableBytes, "GEMM table does not fit");

// The scratch array itself (one copy per device that loads the library).
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoallocBytes];

// Device address of g_noalloc_scratch on the current device (looked up on every call).
dl_status scratch_address(uint8_t **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        set_error("dl_tc_closure_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        return DL_EDEVICE;
    }
    *out = static_cast<uint8_t *>(p);
    return DL_OK;
}

#define NA_CK(x)                                                                               \
    do {                                                                                       \
        const cudaError_t e_ = (x);                                                            \
        if (e_ != cudaSuccess) {                                                               \
            set_error("dl_tc_closure_noalloc: %s: %s", #x, cudaGetErrorString(e_));            \
            return DL_EDEVICE;                                                                 \
        }                                                                                      \
    } while (0)

// Counters and the status word to the host.  A device-side wait that expired (any status bit
// but ST_BAD_INPUT) ends the call at once with DL_ETIMEOUT, so a partial result is never
// mistaken for a non-converged or uncertified closure.
dl_status read_back(cudaStream_t s, const unsigned long long *dev, unsigned long long *host, int count,
                    const int *status, int *status_host) {
    NA_CK(cudaMemcpyAsync(host, dev, sizeof(unsigned long long) * count, cudaMemcpyDeviceToHost, s));
    NA_CK(cudaMemcpyAsync(status_host, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
    if (*status_host & ~ST_BAD_INPUT) {
        set_error("dl_tc_closure_noalloc: a device-side wait expired (status 0x%x)", *status_host);
        return DL_ETIMEOUT;
    }
    return DL_OK;
}

}  // namespace
}  // namespace dl

using namespace dl;

extern "C" DL_API dl_status dl_tc_closure_noalloc(int32_t n, const uint8_t *E, uint64_t *out_bits,
                                                  void *stream, int32_t *squarings) {
    if (squarings) *squarings = 0;
    if (n < 0 || n > kMaxN) {
        set_error("dl_tc_closure_noalloc: n = %d is outside [0, %d], the size its fixed scratch holds",
                  n, static_cast<int>(kMaxN));
        return DL_EINVAL;
    }
    if (n == 0) {  // warm-up: place the array and load every kernel below; writes nothing
        uint8_t *base = nullptr;
        const dl_status rc = scratch_address(&base);
        if (rc) return rc;
        NA_CK(gemm_prepare(KIND_F8, false, 256, EPI_BOOL));
        NA_CK(load_ingest_and_sweep());
        return DL_OK;
    }
    if (!E || !out_bits) {
        set_error("dl_tc_closure_noalloc: E and out_bits must be device pointers, not NULL");
        return DL_EINVAL;
    }
    uint8_t *base = nullptr;
    dl_status rc = scratch_address(&base);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t np = (static_cast<int64_t>(n) + 255) / 256 * 256;
    const int64_t wp = np / 64;
    uint8_t *C0 = base + kOffC0, *C1 = base + kOffC1;
    auto *rbits = reinterpret_cast<uint64_t *>(base + kOffRBits);
    auto *mbits = reinterpret_cast<uint64_t *>(base + kOffMBits);
    auto *table = reinterpret_cast<GemmProblem *>(base + kOffTable);
    auto *scal = reinterpret_cast<unsigned long long *>(base + kOffScalars);  // [0..7]
    int *status = reinterpret_cast<int *>(base + kOffScalars + 1024);
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);

    // counters start at zero on every call: the array still holds the previous call's values
    NA_CK(cudaMemsetAsync(scal, 0, 8 * sizeof(unsigned long long), s));
    NA_CK(cudaMemsetAsync(status, 0, sizeof(int), s));
    NA_CK(ingest_u8_to_e4m3(E, n, static_cast<int>(np), C0, 1, scal + 0, scal + 1, scal + 2, status, s));
    unsigned long long h[8] = {};
    int hst = 0;
    if ((rc = read_back(s, scal, h, 8, status, &hst))) return rc;
    if (hst & ST_BAD_INPUT) {
        set_error("dl_tc_closure_noalloc: E holds a byte that is neither 0 nor 1");
        return DL_EINVAL;
    }
    unsigned long long prev = h[2];

    GemmProblem probs[2];
    std::string err;
    for (int p = 0; p < 2; ++p) {
        const uint8_t *src = p == 0 ? C0 : C1;
        uint8_t *dst = p == 0 ? C1 : C0;
        GemmEpilogue e{};
        e.out8 = dst;
        e.ld_out8 = np;
        e.bits = reinterpret_cast<uint32_t *>(rbits);
        e.ld_bits32 = 2 * wp;
        e.count = scal + 3;
        const Operand op{src, np, np, np, 0, 0};
        if (!gemm_make_problem(&probs[p], KIND_F8, false, 256, static_cast<int>(np), static_cast<int>(np),
                               static_cast<int>(np), op, op, e, &err)) {
            set_error("dl_tc_closure_noalloc: %s", err.c_str());
            return DL_EDEVICE;
        }
    }
    // pageable source: the copy has read it when cudaMemcpyAsync returns
    NA_CK(cudaMemcpyAsync(table, probs, sizeof(probs), cudaMemcpyHostToDevice, s));
    const int tiles = probs[0].tiles_m * probs[0].tiles_n;
    const int grid = std::min(tiles, sms);
    const uint64_t budget = 2000000000ull;
    const int max_squarings = 2 + static_cast<int>(std::ceil(std::log2(static_cast<double>(np) + 1.0)));
    int t = 0;
    bool have_model = false;
    for (;;) {
        if (t >= max_squarings) {
            set_error("dl_tc_closure_noalloc: no convergence in %d squarings", t);
            return DL_ENOTCONV;
        }
        NA_CK(cudaMemsetAsync(scal + 3, 0, sizeof(unsigned long long), s));
        NA_CK(gemm_launch(KIND_F8, false, 256, EPI_BOOL, table + (t & 1), 1, tiles, grid, status, budget, s));
        ++t;
        if ((rc = read_back(s, scal, h, 8, status, &hst))) return rc;
        if (h[3] == prev) break;
        prev = h[3];
        NA_CK(cudaMemsetAsync(scal + 4, 0, 2 * sizeof(unsigned long long), s));
        NA_CK(bits_sweep(E, n, n, rbits, mbits, wp, 0, 1, scal + 4, scal + 5, s));
        if ((rc = read_back(s, scal, h, 8, status, &hst))) return rc;
        if (h[4] == 0) {
            have_model = true;
            break;
        }
    }
    if (!have_model) {
        NA_CK(cudaMemsetAsync(scal + 4, 0, 2 * sizeof(unsigned long long), s));
        NA_CK(bits_sweep(E, n, n, rbits, mbits, wp, 0, 0, scal + 4, scal + 5, s));
        if ((rc = read_back(s, scal, h, 8, status, &hst))) return rc;
        if (h[4] != 0) {
            set_error("dl_tc_closure_noalloc: converged closure failed its certificate");
            return DL_EDEVICE;
        }
    }
    const int64_t w = (n + 63) / 64;
    NA_CK(cudaMemcpy2DAsync(out_bits, w * 8, mbits, wp * 8, w * 8, n, cudaMemcpyDeviceToDevice, s));
    NA_CK(cudaStreamSynchronize(s));
    if (squarings) *squarings = t;
    return DL_OK;
}
