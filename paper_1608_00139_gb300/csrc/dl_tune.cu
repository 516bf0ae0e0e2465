// dl_tune.cu -- the autotuner: for each size bucket (N rounded up to a power of two, at least 256),
// measured choices that the solvers otherwise take from fixed rules:
//   sq_bn         tile width of the FP8 squaring GEMM (128 or 256), the faster on a dense operand;
//   t_sq          seconds per squaring at that width (the AUTO path's cost model, instead of a
//                 flop rate and a launch constant);
//   sweep_rate    bytes per second of an unsaturated Iteration sweep on the CSR (the cost model's
//                 sweep rate, instead of 6 / 3 TB/s by size): the faster of an ER digraph's and a
//                 heavy-tailed DAG's;
//   mx_reserve    SMs the mixed path's LU leaves to its critical chain (16, 32 or 48), and
//   mx_pairs      how many of its first steps go in units sharing one bulk update (0, a quarter,
//   mx_group      half, three quarters or all of them) and the steps per unit (2 or 4): the
//                 fastest factorisation;
//   sg_iteration  same generation on AUTO: the Iteration on bits (1) or the doubling (0) where the
//                 same one is faster on a random forest and on a heavy-tailed DAG, else the
//                 crossover at Np = 6144 (-1).
// Inputs are synthetic and generated on the device (an integer hash per pair): an operand with
// about half ones, an ER digraph of mean degree 8, a random forest, and a DAG shaped like
// preferential attachment (Zipf-like out-degrees, links skewed toward the earliest nodes).  A
// choice measured on one kind of graph can be wrong for another (a route tuned on forests alone
// doubled the serving stream's p99), hence two kinds where the structure matters.  The table lives in the
// context; with a cache path it is read at dl_create and written after every tuning run, as JSON
// keyed by "<GPU name>|<driver version>|<bucket>", so another process on the same kind of GPU
// and driver reuses it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cctype>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "dl_ctx.h"
#include "dl_internal.h"

namespace dl {

namespace {

#define TCK(x)                                                                               \
    do {                                                                                     \
        cudaError_t e_ = (x);                                                                \
        if (e_ != cudaSuccess) {                                                             \
            set_error("autotune: %s failed: %s", #x, cudaGetErrorString(e_));                \
            return DL_EDEVICE;                                                               \
        }                                                                                    \
    } while (0)

__device__ __forceinline__ uint64_t hash64(uint64_t z) {  // SplitMix64's output function
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// e4m3 operand (np x np) with about half ones inside n x n, zero padding.
__global__ void dense_operand_kernel(uint8_t *C, int n, int np, uint64_t seed) {
    const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (t >= static_cast<int64_t>(np) * np) return;
    const int64_t i = t / np, j = t % np;
    C[t] = (i < n && j < n && (hash64(seed + static_cast<uint64_t>(t)) & 1)) ? 0x38 : 0;
}

// ER digraph bytes (n x n): an edge with probability about deg / n, no self-loops.
__global__ void er_bytes_kernel(uint8_t *E, int n, double deg, uint64_t seed) {
    const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (t >= static_cast<int64_t>(n) * n) return;
    const int64_t i = t / n, j = t % n;
    const double u = static_cast<double>(hash64(seed + static_cast<uint64_t>(t)) >> 11) * 0x1.0p-53;
    E[t] = (i != j && u < deg / n) ? 1 : 0;
}

// A random forest as P[i][parent(i)] = 1 (parent uniform below i, roots with probability 1/20).
__global__ void forest_bytes_kernel(uint8_t *P, int n, uint64_t seed) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || i == 0) return;
    const uint64_t h = hash64(seed + static_cast<uint64_t>(i));
    if (h % 20 == 0) return;
    P[static_cast<int64_t>(i) * n + static_cast<int64_t>((h >> 8) % static_cast<uint64_t>(i))] = 1;
}

// A DAG shaped like preferential attachment (the serving workload): node i >= 1 links to
// k = min(i, floor(1 / u)) earlier nodes (a Zipf(2)-like out-degree, heavy-tailed rows; at most
// 4096), each j = floor(i v^3), skewed toward the earliest nodes (hubs).  E zeroed by the caller.
__global__ void skewed_dag_kernel(uint8_t *E, int n, uint64_t seed) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || i == 0) return;
    const double u = static_cast<double>((hash64(seed + static_cast<uint64_t>(i)) >> 11) + 1) * 0x1.0p-53;
    const int k = static_cast<int>(fmin(fmin(static_cast<double>(i), 4096.0), fmax(1.0, floor(1.0 / u))));
    uint8_t *row = E + static_cast<int64_t>(i) * n;
    for (int t = 0; t < k; ++t) {
        const double v =
            static_cast<double>(hash64((seed ^ 0x9E3779B97F4A7C15ull) + (static_cast<uint64_t>(i) << 24) + t) >> 11) *
            0x1.0p-53;
        row[static_cast<int>(fmin(static_cast<double>(i - 1), floor(static_cast<double>(i) * v * v * v)))] = 1;
    }
}

unsigned blocks_for(int64_t count) { return static_cast<unsigned>((count + 255) / 256); }

// ---- JSON cache ---------------------------------------------------------------------------

struct JVal {
    enum Kind { NUM, STR, OBJ } kind = NUM;
    double num = 0;
    std::string str;
    std::vector<std::pair<std::string, JVal>> obj;
};

struct JParser {
    const std::string &t;
    size_t p = 0;
    void ws() {
        while (p < t.size() && std::isspace(static_cast<unsigned char>(t[p]))) ++p;
    }
    bool str(std::string *out) {
        ws();
        if (p >= t.size() || t[p] != '"') return false;
        ++p;
        out->clear();
        while (p < t.size() && t[p] != '"') {
            if (t[p] == '\\' && p + 1 < t.size()) ++p;
            out->push_back(t[p++]);
        }
        if (p >= t.size()) return false;
        ++p;
        return true;
    }
    bool val(JVal *v) {
        ws();
        if (p >= t.size()) return false;
        if (t[p] == '{') {
            ++p;
            v->kind = JVal::OBJ;
            ws();
            if (p < t.size() && t[p] == '}') {
                ++p;
                return true;
            }
            for (;;) {
                std::string k;
                JVal x;
                if (!str(&k)) return false;
                ws();
                if (p >= t.size() || t[p] != ':') return false;
                ++p;
                if (!val(&x)) return false;
                v->obj.emplace_back(k, std::move(x));
                ws();
                if (p < t.size() && t[p] == ',') {
                    ++p;
                    continue;
                }
                if (p < t.size() && t[p] == '}') {
                    ++p;
                    return true;
                }
                return false;
            }
        }
        if (t[p] == '"') {
            v->kind = JVal::STR;
            return str(&v->str);
        }
        char *end = nullptr;
        v->kind = JVal::NUM;
        v->num = std::strtod(t.c_str() + p, &end);
        if (end == t.c_str() + p) return false;
        p = static_cast<size_t>(end - t.c_str());
        return true;
    }
};

const JVal *field(const JVal &o, const char *k) {
    for (auto &kv : o.obj)
        if (kv.first == k) return &kv.second;
    return nullptr;
}

std::string entry_json(const TuneEntry &e) {
    char buf[256];
    std::snprintf(buf, sizeof buf,
                  "{\"sq_bn\": %d, \"t_sq_us\": %.3f, \"sweep_gbs\": %.3f, \"mx_reserve\": %d, \"mx_pairs\": %d, "
                  "\"mx_group\": %d, \"sg_iteration\": %d}",
                  e.sq_bn, e.t_sq * 1e6, e.sweep_rate * 1e-9, e.mx_reserve, e.mx_pairs, e.mx_group, e.sg_iteration);
    return buf;
}

bool entry_from(const JVal &o, TuneEntry *e) {
    if (o.kind != JVal::OBJ) return false;
    const JVal *a = field(o, "sq_bn"), *b = field(o, "t_sq_us"), *c = field(o, "sweep_gbs"),
               *d = field(o, "mx_reserve"), *f = field(o, "sg_iteration");
    if (!a || !b || !c || !d || !f) return false;
    e->sq_bn = static_cast<int>(a->num) == 128 ? 128 : 256;
    e->t_sq = b->num * 1e-6;
    e->sweep_rate = c->num * 1e9;
    e->mx_reserve = std::max(1, static_cast<int>(d->num));
    e->sg_iteration = static_cast<int>(f->num);
    const JVal *g = field(o, "mx_pairs");  // absent in older caches: the default
    e->mx_pairs = g ? static_cast<int>(g->num) : -1;
    const JVal *h = field(o, "mx_group");
    e->mx_group = h && static_cast<int>(h->num) == 4 ? 4 : 2;
    e->measured = true;
    return true;
}

// All entries of a cache file (any GPU), as raw JSON objects by key.
std::map<std::string, std::string> read_cache(const std::string &path, std::map<std::string, TuneEntry> *parsed) {
    std::map<std::string, std::string> raw;
    std::ifstream f(path);
    if (!f) return raw;
    std::stringstream ss;
    ss << f.rdbuf();
    const std::string text = ss.str();
    JParser jp{text};
    JVal root;
    if (!jp.val(&root) || root.kind != JVal::OBJ) return raw;
    const JVal *entries = field(root, "entries");
    if (!entries || entries->kind != JVal::OBJ) return raw;
    for (auto &kv : entries->obj) {
        TuneEntry e;
        if (!entry_from(kv.second, &e)) continue;
        raw[kv.first] = entry_json(e);
        if (parsed) (*parsed)[kv.first] = e;
    }
    return raw;
}

bool write_cache(const std::string &path, const std::map<std::string, std::string> &raw) {
    const std::string tmp = path + ".tmp";
    {
        std::ofstream f(tmp);
        if (!f) return false;
        f << "{\"version\": 1, \"entries\": {";
        bool first = true;
        for (auto &kv : raw) {
            f << (first ? "\n  " : ",\n  ") << '"' << kv.first << "\": " << kv.second;
            first = false;
        }
        f << "\n}}\n";
        if (!f) return false;
    }
    return std::rename(tmp.c_str(), path.c_str()) == 0;
}

std::string key_of(const dl_ctx *ctx, int bucket) { return ctx->tune.key_prefix + std::to_string(bucket); }

// Median of three timed runs of f (CUDA events on s), after one warm-up run.
template <class F>
dl_status time_median(cudaStream_t s, cudaEvent_t a, cudaEvent_t b, F &&f, double *sec) {
    dl_status rc = f();
    if (rc) return rc;
    double t[3];
    for (double &x : t) {
        TCK(cudaEventRecord(a, s));
        if ((rc = f())) return rc;
        TCK(cudaEventRecord(b, s));
        TCK(cudaEventSynchronize(b));
        float ms = 0;
        TCK(cudaEventElapsedTime(&ms, a, b));
        x = ms * 1e-3;
    }
    std::sort(t, t + 3);
    *sec = t[1];
    return DL_OK;
}

}  // namespace

int tune_bucket(int64_t np) {
    int b = 256;
    while (b < np && b < (1 << 20)) b <<= 1;
    return b;
}

TuneEntry tuned(dl_ctx *ctx, int64_t np) {
    const int b = tune_bucket(np);
    std::lock_guard<std::mutex> lk(ctx->tune.mu);
    auto it = ctx->tune.by_bucket.find(b);
    if (it != ctx->tune.by_bucket.end()) return it->second;
    TuneEntry e;
    e.bucket = b;
    return e;
}

void tune_init(dl_ctx *ctx) {
    cudaDeviceProp prop{};
    int drv = 0;
    cudaGetDeviceProperties(&prop, ctx->device);
    cudaDriverGetVersion(&drv);
    std::string name = prop.name;
    for (char &c : name)
        if (c == '"' || c == '\\' || c == '|') c = '_';
    ctx->tune.key_prefix = name + "|" + std::to_string(drv) + "|";
    ctx->tune.autotune = ctx->cfg.autotune != 0;
    const char *path = ctx->cfg.tune_cache ? ctx->cfg.tune_cache : std::getenv("DL_TUNE_CACHE");
    if (path && *path) ctx->tune.cache_path = path;
    if (ctx->tune.cache_path.empty()) return;
    std::map<std::string, TuneEntry> parsed;
    read_cache(ctx->tune.cache_path, &parsed);
    std::lock_guard<std::mutex> lk(ctx->tune.mu);
    for (auto &kv : parsed) {
        if (kv.first.compare(0, ctx->tune.key_prefix.size(), ctx->tune.key_prefix) != 0) continue;
        const int b = std::atoi(kv.first.c_str() + ctx->tune.key_prefix.size());
        if (b < 256) continue;
        TuneEntry e = kv.second;
        e.bucket = b;
        ctx->tune.by_bucket[b] = e;
    }
}

dl_status autotune_bucket(dl_ctx *ctx, Workspace &ws, cudaStream_t s, int32_t n_req, bool force, TuneEntry *out,
                          std::string *source) {
    const int b = tune_bucket((std::max<int64_t>(n_req, 1) + 255) / 256 * 256);
    {
        std::lock_guard<std::mutex> lk(ctx->tune.mu);
        auto it = ctx->tune.by_bucket.find(b);
        if (!force && it != ctx->tune.by_bucket.end() && it->second.measured) {
            *out = it->second;
            *source = "cache";
            return DL_OK;
        }
    }
    TuneEntry e;
    e.bucket = b;
    if (b > 16384) {  // measured only up to N = 16384 (a few GB of scratch); larger sizes keep the rules
        *out = e;
        *source = "defaults (bucket above 16384)";
        return DL_OK;
    }
    const int n = b, np = b;
    const int64_t wp = np / 64, nn = static_cast<int64_t>(np) * np;
    Range trace_("autotune");
    cudaEvent_t ea = ws.ev[0], eb = ws.ev[1];
    // 1. the FP8 squaring at both tile widths
    auto *C = static_cast<uint8_t *>(ws.get("tn_c", nn));
    auto *O = static_cast<uint8_t *>(ws.get("tn_o", nn));
    auto *bits = static_cast<uint64_t *>(ws.get("tn_bits", np * wp * 8));
    if (!C || !O || !bits) {
        set_error("autotune: device allocation failed");
        return DL_ENOMEM;
    }
    dense_operand_kernel<<<blocks_for(nn), 256, 0, s>>>(C, n, np, 0x5eedull);
    TCK(cudaGetLastError());
    TCK(cudaMemsetAsync(ws.status, 0, sizeof(int), s));
    double best = 1e30;
    for (int bn : {128, 256}) {
        GemmEpilogue epi{};
        epi.out8 = O;
        epi.ld_out8 = np;
        epi.bits = reinterpret_cast<uint32_t *>(bits);
        epi.ld_bits32 = 2 * wp;
        epi.count = ws.scal + SC_STEP0;
        GemmProblem pr;
        std::string err;
        const Operand op{C, np, np, np, 0, 0};
        if (!gemm_make_problem(&pr, KIND_F8, false, bn, np, np, np, op, op, epi, &err)) {
            set_error("autotune: %s", err.c_str());
            return DL_EDEVICE;
        }
        auto *d = static_cast<GemmProblem *>(ws.get(bn == 128 ? "tn_p128" : "tn_p256", sizeof(GemmProblem)));
        if (!d) {
            set_error("autotune: device allocation failed");
            return DL_ENOMEM;
        }
        TCK(cudaMemcpyAsync(d, &pr, sizeof pr, cudaMemcpyHostToDevice, s));
        TCK(gemm_prepare(KIND_F8, false, bn, EPI_BOOL));
        const int tiles = pr.tiles_m * pr.tiles_n;
        double t = 0;
        dl_status rc = time_median(s, ea, eb, [&]() -> dl_status {
            TCK(gemm_launch(KIND_F8, false, bn, EPI_BOOL, d, 1, tiles, std::min(tiles, ctx->sms), ws.status,
                            ctx->budget_ns, s));
            return DL_OK;
        }, &t);
        if (rc) return rc;
        if (t < best) {
            best = t;
            e.sq_bn = bn;
        }
    }
    e.t_sq = best;
    // 2. an unsaturated Iteration sweep (the emission E M, which changes nothing in place), on an
    // ER digraph of mean degree 8 and on the skewed DAG (heavy-tailed rows); the faster rate is
    // kept, so that the cost model does not square a graph whose sweeps are cheap
    auto *E = static_cast<uint8_t *>(ws.get("tn_e", static_cast<size_t>(n) * n));
    auto *D = static_cast<uint8_t *>(ws.get("tn_d", static_cast<size_t>(n) * n));
    auto *cnt = static_cast<int *>(ws.get("tn_cnt", (np + 1) * 4));
    auto *ptr = static_cast<int *>(ws.get("tn_ptr", (np + 1) * 4));
    auto *uoff = static_cast<int *>(ws.get("tn_units", (np + 1) * 4));
    auto *colmask = static_cast<uint64_t *>(ws.get("tn_colmask", wp * 8));
    auto *M = static_cast<uint64_t *>(ws.get("tn_m", np * wp * 8));
    if (!E || !D || !cnt || !ptr || !uoff || !colmask || !M) {
        set_error("autotune: device allocation failed");
        return DL_ENOMEM;
    }
    er_bytes_kernel<<<blocks_for(static_cast<int64_t>(n) * n), 256, 0, s>>>(E, n, 8.0, 0xe5eedull);
    TCK(cudaGetLastError());
    TCK(cudaMemsetAsync(D, 0, static_cast<size_t>(n) * n, s));
    skewed_dag_kernel<<<blocks_for(n), 256, 0, s>>>(D, n, 0xda9ull);
    TCK(cudaGetLastError());
    dl_status rc = DL_OK;
    auto sweep_rate = [&](const uint8_t *G, double *rate) -> dl_status {
        TCK(cudaMemsetAsync(ws.scal, 0, kScalars * sizeof(unsigned long long), s));
        TCK(cudaMemsetAsync(colmask, 0, wp * 8, s));
        TCK(csr_pack_checked(G, n, np, wp, cnt, ptr, M, ws.scal + SC_DMAX, ws.scal + SC_NNZ, ws.scal + SC_COUNT0,
                             ws.status, colmask, s));
        unsigned long long hs[2] = {0, 0};
        TCK(cudaMemcpyAsync(hs, ws.scal + SC_DMAX, sizeof hs, cudaMemcpyDeviceToHost, s));  // dmax, nnz
        TCK(cudaStreamSynchronize(s));
        auto *col = static_cast<int *>(ws.get("tn_col", std::max<size_t>(hs[1] + static_cast<size_t>(n), 1) * 4));
        if (!col) {
            set_error("autotune: device allocation failed");
            return DL_ENOMEM;
        }
        TCK(csr_fill_from_bits(M, n, wp, ptr, col, s));
        TCK(sweep_units(ptr, n, cnt, uoff, s));
        double tsw = 0;
        dl_status r2 = time_median(s, ea, eb, [&]() -> dl_status {
            int launches = 0;
            TCK(bits_sweep_csr(ptr, col, uoff, n, M, bits, wp, 0, ws.scal + SC_VIOL, ws.scal + SC_ONES, &launches, s,
                               static_cast<int>(hs[0])));
            return DL_OK;
        }, &tsw);
        if (r2) return r2;
        const double nnz_i = static_cast<double>(hs[1]) + n;  // the CSR of I + G
        *rate = (nnz_i * wp * 8 + 2.0 * np * wp * 8) / std::max(tsw, 1e-7);
        return DL_OK;
    };
    double rate_er = 0, rate_dag = 0;
    if ((rc = sweep_rate(E, &rate_er)) || (rc = sweep_rate(D, &rate_dag))) return rc;
    e.sweep_rate = std::max(rate_er, rate_dag);
    // 3. the mixed path's reserve and 4. the same-generation route, through the solvers themselves
    auto *ob = static_cast<uint64_t *>(ws.get("tn_out", static_cast<size_t>(n) * ((n + 63) / 64) * 8));
    if (!ob) {
        set_error("autotune: device allocation failed");
        return DL_ENOMEM;
    }
    auto set_entry = [&](const TuneEntry &x) {
        std::lock_guard<std::mutex> lk(ctx->tune.mu);
        ctx->tune.by_bucket[b] = x;
    };
    if (np >= 2048) {  // coordinate search: the reserve at the default pairing, then the pairing
        auto factor_ms = [&](const TuneEntry &x, double *ms) -> dl_status {
            set_entry(x);
            SolveArgs a;
            a.n = n;
            a.E = E;
            a.mem = DL_MEM_DEVICE;
            a.path = DL_PATH_MIXED;
            a.out_bits = ob;
            for (int rep = 0; rep < 2; ++rep) {  // the second run's factorisation time
                dl_stats st{};
                dl_status r2 = solve_tc(ctx, ws, s, a, &st);
                if (r2) return r2;
                *ms = st.ms_factor;
            }
            return DL_OK;
        };
        double best_f = 1e30;
        for (int r : {16, 32, 48}) {
            TuneEntry x = e;
            x.mx_reserve = r;
            double ms = 0;
            if ((rc = factor_ms(x, &ms))) return rc;
            if (ms < best_f) {
                best_f = ms;
                e.mx_reserve = r;
            }
        }
        const int nb = np / 128;
        for (int group : {2, 4}) {
            for (int grouped : {0, nb / 4, nb / 2, 3 * nb / 4, nb}) {
                if (group == 2 && grouped == nb / 2) continue;  // the default, measured above
                if (group == 4 && grouped == 0) continue;        // the same as no grouping
                TuneEntry x = e;
                x.mx_group = group;
                x.mx_pairs = grouped;
                double ms = 0;
                if ((rc = factor_ms(x, &ms))) return rc;
                if (ms < best_f) {
                    best_f = ms;
                    e.mx_group = group;
                    e.mx_pairs = grouped;
                }
            }
        }
    }
    {  // the same-generation route: a choice only where one route wins on both a random forest
       // and the skewed DAG (their relations differ widely in depth and density), else the rule
        auto *P = E;  // reuses the ER graph's bytes
        TCK(cudaMemsetAsync(P, 0, static_cast<size_t>(n) * n, s));
        forest_bytes_kernel<<<blocks_for(n), 256, 0, s>>>(P, n, 0xf0e5ull);
        TCK(cudaGetLastError());
        int pick[2] = {-1, -1};
        const uint8_t *graphs[2] = {P, D};
        for (int gi = 0; gi < 2; ++gi) {
            double best_s = 1e30;
            for (int it : {0, 1}) {
                TuneEntry x = e;
                x.sg_iteration = it;
                set_entry(x);
                SolveArgs a;
                a.n = n;
                a.E = graphs[gi];
                a.mem = DL_MEM_DEVICE;
                a.path = DL_PATH_AUTO;
                a.out_bits = ob;
                double t = 0;
                for (int rep = 0; rep < 2; ++rep) {
                    dl_stats st{};
                    if ((rc = solve_sg(ctx, ws, s, a, &st))) return rc;
                    t = st.ms_total;
                }
                if (t < best_s) {
                    best_s = t;
                    pick[gi] = it;
                }
            }
        }
        e.sg_iteration = pick[0] == pick[1] ? pick[0] : -1;
    }
    e.measured = true;
    set_entry(e);
    *out = e;
    *source = "measured";
    if (!ctx->tune.cache_path.empty()) {
        std::map<std::string, std::string> raw = read_cache(ctx->tune.cache_path, nullptr);
        raw[key_of(ctx, b)] = entry_json(e);
        if (!write_cache(ctx->tune.cache_path, raw)) {
            set_error("autotune: cannot write the cache file %s", ctx->tune.cache_path.c_str());
            return DL_EINVAL;
        }
    }
    return DL_OK;
}

std::string tune_report(const dl_ctx *ctx, const TuneEntry &e, const std::string &source) {
    std::ostringstream o;
    o << "{\"key\": \"" << key_of(ctx, e.bucket) << "\", \"bucket\": " << e.bucket << ", \"source\": \"" << source
      << "\", \"entry\": " << entry_json(e) << "}";
    return o.str();
}

}  // namespace dl
