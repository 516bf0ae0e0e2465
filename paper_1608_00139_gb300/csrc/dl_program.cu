// dl_program.cu -- the program front-end: a linear Datalog program over binary predicates
// (the class C_lin of Sec. 5), evaluated layer by layer on the library's solvers.
//
//  * Parsing.  Clauses  head(X,Y) :- a1(..), ..., ak(..).  with variables only (an identifier that
//    starts with an upper-case letter or '_'), every predicate binary, "not p(X,Y)" for a negated
//    atom.  Base relations (predicates that head no clause) are given as n x n 0/1 matrices.
//  * C_lin (Sec. 5).  A body must be a chain X = x0 - x1 - ... - xk = Y between the head's two
//    variables, every atom joining two consecutive variables in either orientation and no variable
//    repeated; it is then the matrix product of its atoms' matrices, an atom read backwards being
//    the transpose (Sec. 2: a conjunction is a product, the existential variables are summed).
//    Linear: no body holds two predicates of the head's strongly connected component (SCC).
//  * Layers.  Predicates depend on the predicates of their clauses' bodies; Tarjan's algorithm
//    gives the SCCs, which are evaluated in a topological order (the layers DB'_1 .. DB'_L of
//    Sec. 5).  A negated atom must name a predicate of a lower layer (stratified negation); its
//    matrix is 1 - R.
//  * A layer's equations (eq. matrixeq:gen0).  Each clause of r_h gives a term: A (no recursive
//    atom), or B R_j C (B, C the products of the atoms before and after the recursive atom R_j,
//    which may be read transposed).  The layer is solved by the first rule that applies:
//      - no recursive term: R_h = min1(sum A);
//      - every recursive term B R_j (C = I, not transposed): the tail recursive class (Sec. 6.1);
//        one equation by dl_tail_recursive's boolean route, several by one closure of the
//        stacked system (the least solution of R = min1(A + B R) over m n constants);
//      - every recursive term R_j C (B = I): the same on the transposes;
//      - one equation, every recursive term B R^T: the transposed class (Sec. 6.2) through the
//        two-sided reduction R = min1(A + B A^T + B R B^T);
//      - one equation, one term B R B^T: the same-generation solver (Sec. 6.3 / 7.2);
//      - otherwise the series of Lemma 3 (eq. series:gen), R^(k+1) = min1(F[R^(k)]) from 0, on
//        FP8 products until nothing changes (this covers mutually recursive two-sided layers,
//        for which the paper gives no linear-algebraic solver).
//  All relations live on the device as n x n 0/1 bytes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cctype>
#include <cstring>
#include <functional>
#include <map>
#include <set>
#include <sstream>
#include <string>
#include <vector>

#include "dl_ctx.h"
#include "dl_internal.h"

namespace dl {

struct PAtom {
    std::string pred;
    int a = 0, b = 0;  // variable ids
    bool neg = false;
};

struct PClause {
    std::string head;
    int ha = 0, hb = 0;
    std::vector<PAtom> body;
    std::string text;
};

// One factor of a chain: a relation, read transposed and/or complemented.
struct Factor {
    std::string pred;
    bool transposed = false, negated = false;
};

}  // namespace dl

struct dl_program {
    dl_ctx *ctx = nullptr;
    std::vector<dl::PClause> clauses;
    std::set<std::string> idb, edb;
    std::vector<std::vector<std::string>> layers;  // topological order
    std::map<std::string, int> layer_of;
    std::map<std::string, uint8_t *> rel;  // device n x n bytes
    int32_t n = -1;                         // size of the relations set so far
    std::string plan;                       // the last run's layer-by-layer account
    bool ran = false;
};

namespace dl {

namespace {

#define PCK(x)                                                                                   \
    do {                                                                                         \
        cudaError_t e_ = (x);                                                                    \
        if (e_ != cudaSuccess) {                                                                 \
            set_error("program: %s failed: %s", #x, cudaGetErrorString(e_));                    \
            return DL_EDEVICE;                                                                   \
        }                                                                                        \
    } while (0)

// ---- parsing ----------------------------------------------------------------------------------

struct Lexer {
    const char *p;
    std::string tok;
    bool next() {
        while (*p && std::isspace(static_cast<unsigned char>(*p))) ++p;
        if (*p == '%') {  // comment to the end of the line
            while (*p && *p != '\n') ++p;
            return next();
        }
        if (!*p) return false;
        if (std::isalpha(static_cast<unsigned char>(*p)) || *p == '_') {
            const char *q = p;
            while (std::isalnum(static_cast<unsigned char>(*q)) || *q == '_') ++q;
            tok.assign(p, q);
            p = q;
            return true;
        }
        if (p[0] == ':' && p[1] == '-') {
            tok = ":-";
            p += 2;
            return true;
        }
        tok.assign(p, 1);
        ++p;
        return true;
    }
};

bool is_var(const std::string &t) { return !t.empty() && (std::isupper(static_cast<unsigned char>(t[0])) || t[0] == '_'); }

dl_status parse(const char *text, std::vector<PClause> *out) {
    Lexer lx{text, {}};
    auto fail = [&](const std::string &why) {
        set_error("program: %s (near \"%s\")", why.c_str(), lx.tok.c_str());
        return DL_EINVAL;
    };
    while (lx.next()) {
        PClause c;
        std::map<std::string, int> vars;
        auto var_id = [&](const std::string &v) {
            auto it = vars.find(v);
            if (it != vars.end()) return it->second;
            const int id = static_cast<int>(vars.size());
            vars[v] = id;
            return id;
        };
        const char *start = lx.p - lx.tok.size();
        auto atom = [&](PAtom *at, bool allow_not) -> dl_status {
            if (allow_not && lx.tok == "not") {
                at->neg = true;
                if (!lx.next()) return fail("unexpected end after 'not'");
            }
            if (is_var(lx.tok) || !(std::isalpha(static_cast<unsigned char>(lx.tok[0])) || lx.tok[0] == '_'))
                return fail("expected a predicate name");
            at->pred = lx.tok;
            std::string v1, v2;
            if (!lx.next() || lx.tok != "(") return fail("expected '('");
            if (!lx.next() || !is_var(lx.tok)) return fail("expected a variable (constants are not allowed)");
            v1 = lx.tok;
            if (!lx.next() || lx.tok != ",") return fail("every predicate must be binary");
            if (!lx.next() || !is_var(lx.tok)) return fail("expected a variable (constants are not allowed)");
            v2 = lx.tok;
            if (!lx.next() || lx.tok != ")") return fail("every predicate must be binary");
            at->a = var_id(v1);
            at->b = var_id(v2);
            return DL_OK;
        };
        PAtom h;
        dl_status rc = atom(&h, false);
        if (rc) return rc;
        c.head = h.pred;
        c.ha = h.a;
        c.hb = h.b;
        if (!lx.next() || lx.tok != ":-") return fail("expected ':-' (facts come in as base relations)");
        for (;;) {
            if (!lx.next()) return fail("unexpected end of the program");
            PAtom at;
            if ((rc = atom(&at, true))) return rc;
            c.body.push_back(at);
            if (!lx.next()) return fail("missing '.'");
            if (lx.tok == ".") break;
            if (lx.tok != ",") return fail("expected ',' or '.'");
        }
        c.text.assign(start, lx.p);
        out->push_back(std::move(c));
    }
    if (out->empty()) {
        set_error("program: no clauses");
        return DL_EINVAL;
    }
    return DL_OK;
}

// The body as a chain from the head's first variable to its second: the factors in order.
dl_status chain_of(const PClause &c, std::vector<Factor> *out) {
    if (c.ha == c.hb) {
        set_error("program: the head of \"%s\" repeats a variable (C_lin needs two different ones)", c.text.c_str());
        return DL_EINVAL;
    }
    std::vector<bool> used(c.body.size(), false);
    std::set<int> seen{c.ha};
    int cur = c.ha;
    for (size_t step = 0; step < c.body.size(); ++step) {
        int pick = -1;
        for (size_t k = 0; k < c.body.size(); ++k) {
            if (used[k] || (c.body[k].a != cur && c.body[k].b != cur)) continue;
            if (pick >= 0) {
                set_error("program: the body of \"%s\" branches at a variable (not a chain)", c.text.c_str());
                return DL_EINVAL;
            }
            pick = static_cast<int>(k);
        }
        if (pick < 0) {
            set_error("program: the body of \"%s\" is not a chain between the head's variables", c.text.c_str());
            return DL_EINVAL;
        }
        const PAtom &at = c.body[pick];
        used[pick] = true;
        if (at.a == at.b) {
            set_error("program: an atom of \"%s\" repeats a variable", c.text.c_str());
            return DL_EINVAL;
        }
        Factor f{at.pred, at.a != cur, at.neg};
        cur = at.a == cur ? at.b : at.a;
        if (!seen.insert(cur).second) {
            set_error("program: the body of \"%s\" revisits a variable (not a chain)", c.text.c_str());
            return DL_EINVAL;
        }
        out->push_back(f);
    }
    if (cur != c.hb) {
        set_error("program: the body of \"%s\" does not end at the head's second variable", c.text.c_str());
        return DL_EINVAL;
    }
    return DL_OK;
}

// Tarjan's strongly connected components of the predicate dependency graph; components come out
// in reverse topological order (a component after every component it depends on).
void tarjan(const std::vector<std::string> &nodes, const std::map<std::string, std::set<std::string>> &succ,
            std::vector<std::vector<std::string>> *comps) {
    std::map<std::string, int> index, low;
    std::set<std::string> on;
    std::vector<std::string> stack;
    int counter = 0;
    std::function<void(const std::string &)> visit = [&](const std::string &v) {
        index[v] = low[v] = counter++;
        stack.push_back(v);
        on.insert(v);
        auto it = succ.find(v);
        if (it != succ.end())
            for (const std::string &w : it->second) {
                if (!index.count(w)) {
                    visit(w);
                    low[v] = std::min(low[v], low[w]);
                } else if (on.count(w)) {
                    low[v] = std::min(low[v], index[w]);
                }
            }
        if (low[v] == index[v]) {
            std::vector<std::string> comp;
            for (;;) {
                const std::string w = stack.back();
                stack.pop_back();
                on.erase(w);
                comp.push_back(w);
                if (w == v) break;
            }
            std::sort(comp.begin(), comp.end());
            comps->push_back(comp);
        }
    };
    for (const std::string &v : nodes)
        if (!index.count(v)) visit(v);
}

// ---- device helpers ---------------------------------------------------------------------------

__global__ void transpose_u8_kernel(const uint8_t *__restrict__ src, int n, uint8_t *__restrict__ dst) {
    __shared__ uint8_t tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int r = r0 + y, c = c0 + threadIdx.x;
        if (r < n && c < n) tile[y][threadIdx.x] = src[static_cast<int64_t>(r) * n + c];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int r = c0 + y, c = r0 + threadIdx.x;
        if (r < n && c < n) dst[static_cast<int64_t>(r) * n + c] = tile[threadIdx.x][y];
    }
}

__global__ void or_u8_kernel(uint8_t *__restrict__ dst, const uint8_t *__restrict__ src, int64_t count) {
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < count;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x)
        dst[t] |= src[t];
}

__global__ void complement_u8_kernel(const uint8_t *__restrict__ src, int64_t count, uint8_t *__restrict__ dst) {
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < count;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x)
        dst[t] = src[t] ? 0 : 1;
}

__global__ void differ_u8_kernel(const uint8_t *__restrict__ a, const uint8_t *__restrict__ b, int64_t count,
                                 unsigned long long *diff) {
    unsigned long long d = 0;
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < count;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x)
        d += a[t] != b[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if ((threadIdx.x & 31) == 0 && d) atomicAdd(diff, d);
}

unsigned grid_for(int64_t count) { return static_cast<unsigned>(std::min<int64_t>((count + 255) / 256, 8192)); }

// Relations of one run: device byte matrices owned by the run (freed at its end).
struct Pool {
    std::vector<void *> owned;
    ~Pool() {
        for (void *p : owned) cudaFree(p);
    }
    uint8_t *alloc(size_t bytes) {
        void *p = nullptr;
        if (device_alloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) return nullptr;
        owned.push_back(p);
        return static_cast<uint8_t *>(p);
    }
};

struct Runner {
    dl_ctx *ctx;
    Workspace &ws;
    cudaStream_t s;
    int32_t n;
    Pool *pool;
    int gemms = 0, launches = 0;
    double ms = 0.0;

    int64_t nn() const { return static_cast<int64_t>(n) * n; }

    dl_status mat(uint8_t **out) {
        *out = pool->alloc(static_cast<size_t>(nn()));
        if (!*out) {
            set_error("program: device allocation failed");
            return DL_ENOMEM;
        }
        return DL_OK;
    }
    dl_status transpose(const uint8_t *a, uint8_t **out) {
        dl_status rc = mat(out);
        if (rc) return rc;
        dim3 grid(static_cast<unsigned>((n + 31) / 32), static_cast<unsigned>((n + 31) / 32));
        transpose_u8_kernel<<<grid, dim3(32, 8), 0, s>>>(a, n, *out);
        PCK(cudaGetLastError());
        ++launches;
        return DL_OK;
    }
    dl_status complement(const uint8_t *a, uint8_t **out) {
        dl_status rc = mat(out);
        if (rc) return rc;
        complement_u8_kernel<<<grid_for(nn()), 256, 0, s>>>(a, nn(), *out);
        PCK(cudaGetLastError());
        ++launches;
        return DL_OK;
    }
    dl_status or_into(uint8_t *dst, const uint8_t *src) {
        or_u8_kernel<<<grid_for(nn()), 256, 0, s>>>(dst, src, nn());
        PCK(cudaGetLastError());
        ++launches;
        return DL_OK;
    }
    dl_status zero(uint8_t **out) {
        dl_status rc = mat(out);
        if (rc) return rc;
        PCK(cudaMemsetAsync(*out, 0, static_cast<size_t>(nn()), s));
        return DL_OK;
    }
    dl_status identity(uint8_t **out) {
        dl_status rc = zero(out);
        if (rc) return rc;
        PCK(cudaMemset2DAsync(*out, static_cast<size_t>(n) + 1, 1, 1, n, s));  // the diagonal bytes
        return DL_OK;
    }
    dl_status copy(uint8_t *dst, const uint8_t *src) {
        PCK(cudaMemcpyAsync(dst, src, static_cast<size_t>(nn()), cudaMemcpyDeviceToDevice, s));
        return DL_OK;
    }
    // bits (n rows of ceil(n/64) words, device) to bytes
    dl_status unpack(const uint64_t *bits, uint8_t **out) {
        dl_status rc = mat(out);
        if (rc) return rc;
        PCK(unpack_bits_u8(bits, n, *out, ws.status, s));
        ++launches;
        return DL_OK;
    }
    uint64_t *bitbuf() {
        auto *b = static_cast<uint64_t *>(ws.get("pg_bits", static_cast<size_t>(n) * ((n + 63) / 64) * 8 + 16));
        if (!b) set_error("program: device allocation failed");
        return b;
    }
    void account(const dl_stats &st) {
        gemms += st.gemm_launches;
        launches += st.gpu_launches;
        ms += st.ms_total;
    }
    // min1(X Y) on the FP8 tensor cores; null stands for the identity
    dl_status product(const uint8_t *x, const uint8_t *y, uint8_t **out) {
        if (!x || !y) {
            *out = const_cast<uint8_t *>(x ? x : y);
            return DL_OK;
        }
        uint64_t *bits = bitbuf();
        if (!bits) return DL_ENOMEM;
        SolveArgs c;
        c.n = n;
        c.E = x;
        c.E2 = y;
        c.mem = DL_MEM_DEVICE;
        c.out_bits = bits;
        dl_stats st{};
        dl_status rc = solve_compose(ctx, ws, s, c, &st);
        if (rc) return rc;
        account(st);
        return unpack(bits, out);
    }
    // the least solution of R = min1(A + P R P^T) (the same-generation solver) into bytes
    dl_status two_sided(const uint8_t *P, const uint8_t *A, uint8_t **out) {
        uint64_t *bits = bitbuf();
        if (!bits) return DL_ENOMEM;
        SolveArgs a;
        a.n = n;
        a.E = P;
        a.E2 = A;
        a.mem = DL_MEM_DEVICE;
        a.path = DL_PATH_AUTO;
        a.out_bits = bits;
        dl_stats st{};
        dl_status rc = solve_sg(ctx, ws, s, a, &st);
        if (rc) return rc;
        account(st);
        return unpack(bits, out);
    }
    dl_status equal(const uint8_t *a, const uint8_t *b, bool *eq) {
        auto *d = static_cast<unsigned long long *>(ws.get("pg_diff", 16));
        if (!d) {
            set_error("program: device allocation failed");
            return DL_ENOMEM;
        }
        PCK(cudaMemsetAsync(d, 0, sizeof(unsigned long long), s));
        differ_u8_kernel<<<grid_for(nn()), 256, 0, s>>>(a, b, nn(), d);
        PCK(cudaGetLastError());
        ++launches;
        unsigned long long h = 0;
        PCK(cudaMemcpyAsync(&h, d, sizeof h, cudaMemcpyDeviceToHost, s));
        PCK(cudaStreamSynchronize(s));
        *eq = h == 0;
        return DL_OK;
    }
};

// A clause's contribution to its layer: A (no recursive atom) or B R_j^o C.
struct Term {
    bool recursive = false;
    int j = -1;                 // index of R_j in the layer
    bool transposed = false;    // R_j^T
    uint8_t *A = nullptr;       // the whole product (non-recursive)
    uint8_t *B = nullptr, *C = nullptr;  // null = identity
};

}  // namespace

dl_status program_create(dl_ctx *ctx, const char *text, dl_program **out) {
    auto *p = new (std::nothrow) dl_program;
    if (!p) {
        set_error("program: out of host memory");
        return DL_ENOMEM;
    }
    p->ctx = ctx;
    dl_status rc = parse(text, &p->clauses);
    if (rc) {
        delete p;
        return rc;
    }
    for (const PClause &c : p->clauses) p->idb.insert(c.head);
    std::map<std::string, std::set<std::string>> succ;
    for (const PClause &c : p->clauses) {
        std::vector<Factor> f;
        if ((rc = chain_of(c, &f))) {
            delete p;
            return rc;
        }
        for (const PAtom &a : c.body) {
            if (p->idb.count(a.pred)) succ[c.head].insert(a.pred);
            else p->edb.insert(a.pred);
        }
    }
    std::vector<std::string> nodes(p->idb.begin(), p->idb.end());
    tarjan(nodes, succ, &p->layers);  // every layer after the layers it reads
    for (size_t l = 0; l < p->layers.size(); ++l)
        for (const std::string &r : p->layers[l]) p->layer_of[r] = static_cast<int>(l);
    // linearity and stratification
    for (const PClause &c : p->clauses) {
        const int lh = p->layer_of[c.head];
        int same = 0;
        for (const PAtom &a : c.body) {
            if (!p->idb.count(a.pred) || p->layer_of[a.pred] != lh) continue;
            if (a.neg) {
                set_error("program: \"%s\" negates %s inside its own layer (not stratified)", c.text.c_str(),
                          a.pred.c_str());
                delete p;
                return DL_EINVAL;
            }
            ++same;
        }
        if (same > 1) {
            set_error("program: \"%s\" has %d body atoms of its head's layer (not linear, Sec. 5)", c.text.c_str(),
                      same);
            delete p;
            return DL_EINVAL;
        }
    }
    *out = p;
    return DL_OK;
}

void program_destroy(dl_program *p) {
    if (!p) return;
    for (auto &kv : p->rel) cudaFree(kv.second);
    delete p;
}

dl_status program_set(dl_program *p, cudaStream_t s, const char *pred, int32_t n, const uint8_t *R, dl_mem mem) {
    if (!p->edb.count(pred)) {
        set_error("program: %s is not a base relation of the program", pred);
        return DL_EINVAL;
    }
    if (p->n >= 0 && p->n != n) {
        set_error("program: every relation must have the same n (%d, not %d)", p->n, n);
        return DL_EINVAL;
    }
    const size_t bytes = static_cast<size_t>(n) * n;
    uint8_t *&d = p->rel[pred];
    if (!d && device_alloc(reinterpret_cast<void **>(&d), std::max<size_t>(bytes, 16)) != cudaSuccess) {
        d = nullptr;
        p->rel.erase(pred);
        set_error("program: device allocation failed");
        return DL_ENOMEM;
    }
    PCK(cudaMemcpyAsync(d, R, bytes, mem == DL_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    PCK(cudaStreamSynchronize(s));
    p->n = n;
    p->ran = false;
    return DL_OK;
}

dl_status program_run(dl_ctx *ctx, Workspace &ws, cudaStream_t s, dl_program *p, dl_stats *st) {
    if (p->n < 0) {
        set_error("program: no base relation has been set");
        return DL_EINVAL;
    }
    for (const std::string &e : p->edb)
        if (!p->rel.count(e)) {
            set_error("program: base relation %s has not been set", e.c_str());
            return DL_EINVAL;
        }
    const int32_t n = p->n;
    const size_t nbytes = std::max<size_t>(static_cast<size_t>(n) * n, 16);
    std::ostringstream plan;
    Pool pool;
    Runner R{ctx, ws, s, n, &pool};
    dl_status rc;
    std::map<std::string, uint8_t *> model;  // this run's models (pool-owned until kept)
    if (n > 0) {
        // every base relation holds 0/1 bytes (the ingest's check, on the packing kernel)
        const int64_t np = (static_cast<int64_t>(n) + 255) / 256 * 256, wp = np / 64;
        auto *M = static_cast<uint64_t *>(ws.get("pg_out", static_cast<size_t>(np) * wp * 8));
        if (!M) {
            set_error("program: device allocation failed");
            return DL_ENOMEM;
        }
        PCK(cudaMemsetAsync(ws.status, 0, sizeof(int), s));
        for (const std::string &e : p->edb) {
            PCK(pack_bits(p->rel[e], n, static_cast<int>(np), wp, M, ws.status, s));
            ++R.launches;
        }
        int stw = 0;
        PCK(cudaMemcpyAsync(&stw, ws.status, sizeof stw, cudaMemcpyDeviceToHost, s));
        PCK(cudaStreamSynchronize(s));
        if (stw & ST_BAD_INPUT) {
            set_error("program: a base relation holds a byte that is neither 0 nor 1");
            return DL_EINVAL;
        }
    }
    auto matrix_of = [&](const Factor &f, uint8_t **out) -> dl_status {
        uint8_t *m = p->idb.count(f.pred) ? model[f.pred] : p->rel[f.pred];
        dl_status r2;
        if (f.negated && (r2 = R.complement(m, &m))) return r2;
        if (f.transposed && (r2 = R.transpose(m, &m))) return r2;
        *out = m;
        return DL_OK;
    };
    auto chain_product = [&](const std::vector<Factor> &fs, size_t b, size_t e, uint8_t **out) -> dl_status {
        uint8_t *acc = nullptr;  // identity
        for (size_t k = b; k < e; ++k) {
            uint8_t *m = nullptr;
            dl_status r2 = matrix_of(fs[k], &m);
            if (r2) return r2;
            if ((r2 = R.product(acc, m, &acc))) return r2;
        }
        *out = acc;
        return DL_OK;
    };
    for (size_t l = 0; l < p->layers.size(); ++l) {
        const std::vector<std::string> &preds = p->layers[l];
        const int M = static_cast<int>(preds.size());
        std::map<std::string, int> idx;
        for (int h = 0; h < M; ++h) idx[preds[h]] = h;
        std::vector<uint8_t *> out(M, nullptr);
        std::string how;
        if (n == 0) {
            how = "empty (n = 0)";
        } else {
            // the layer's equations: A_h = OR of the non-recursive clauses' products, and the terms
            std::vector<uint8_t *> A(M, nullptr);
            std::vector<std::vector<Term>> terms(M);
            for (int h = 0; h < M; ++h)
                if ((rc = R.zero(&A[h]))) return rc;
            for (const PClause &c : p->clauses) {
                if (!idx.count(c.head)) continue;
                const int h = idx[c.head];
                std::vector<Factor> fs;
                if ((rc = chain_of(c, &fs))) return rc;
                int rpos = -1;
                for (size_t k = 0; k < fs.size(); ++k)
                    if (idx.count(fs[k].pred)) rpos = static_cast<int>(k);
                Term t;
                if (rpos < 0) {
                    if ((rc = chain_product(fs, 0, fs.size(), &t.A))) return rc;
                    if ((rc = R.or_into(A[h], t.A))) return rc;
                } else {
                    t.recursive = true;
                    t.j = idx[fs[rpos].pred];
                    t.transposed = fs[rpos].transposed;
                    if ((rc = chain_product(fs, 0, rpos, &t.B))) return rc;
                    if ((rc = chain_product(fs, rpos + 1, fs.size(), &t.C))) return rc;
                    terms[h].push_back(t);
                }
            }
            bool any_rec = false, left = true, right = true, trans_left = M == 1, trans_right = M == 1;
            for (int h = 0; h < M; ++h)
                for (const Term &t : terms[h]) {
                    any_rec = true;
                    left = left && !t.transposed && t.C == nullptr;
                    right = right && !t.transposed && t.B == nullptr;
                    trans_left = trans_left && t.transposed && t.C == nullptr;
                    trans_right = trans_right && t.transposed && t.B == nullptr;
                }
            bool sg_form = false;
            if (M == 1 && terms[0].size() == 1 && !terms[0][0].transposed && terms[0][0].B && terms[0][0].C) {
                uint8_t *bt = nullptr;
                if ((rc = R.transpose(terms[0][0].B, &bt)) || (rc = R.equal(bt, terms[0][0].C, &sg_form))) return rc;
            }
            auto tail = [&](int32_t size, const uint8_t *B0, const uint8_t *Aa, uint64_t *bits) -> dl_status {
                SolveArgs a;
                a.n = size;
                a.E = B0;
                a.E2 = Aa;
                a.mem = DL_MEM_DEVICE;
                a.path = DL_PATH_AUTO;
                a.out_bits = bits;
                dl_stats ts{};
                dl_status r2 = solve_tail(ctx, ws, s, a, &ts);
                R.account(ts);
                return r2;
            };
            // OR of the terms' outer coefficients (null = the identity)
            auto coeff_sum = [&](bool use_b, uint8_t **sum) -> dl_status {
                dl_status r2 = R.zero(sum);
                if (r2) return r2;
                for (const Term &t : terms[0]) {
                    uint8_t *c = use_b ? t.B : t.C;
                    if (!c && (r2 = R.identity(&c))) return r2;
                    if ((r2 = R.or_into(*sum, c))) return r2;
                }
                return DL_OK;
            };
            if (!any_rec) {
                how = "non-recursive: R = min1(sum of the clauses' products)";
                out = A;
            } else if (left || right) {
                // right-recursive terms R_j C: solve the transposes, R^T = A^T + sum C^T R_j^T
                std::vector<uint8_t *> Aa(A);
                std::vector<std::vector<uint8_t *>> Bj(M, std::vector<uint8_t *>(M, nullptr));
                for (int h = 0; h < M; ++h) {
                    if (!left && (rc = R.transpose(A[h], &Aa[h]))) return rc;
                    for (const Term &t : terms[h]) {
                        uint8_t *b = left ? t.B : nullptr;
                        if (!left && t.C && (rc = R.transpose(t.C, &b))) return rc;
                        if (!b && (rc = R.identity(&b))) return rc;  // a term R_j alone
                        if (!Bj[h][t.j] && (rc = R.zero(&Bj[h][t.j]))) return rc;
                        if ((rc = R.or_into(Bj[h][t.j], b))) return rc;
                    }
                }
                if (M == 1) {
                    uint8_t *B0 = Bj[0][0];
                    uint64_t *bits = R.bitbuf();
                    if (!bits) return DL_ENOMEM;
                    if ((rc = tail(n, B0, Aa[0], bits))) return rc;
                    if ((rc = R.unpack(bits, &out[0]))) return rc;
                } else {  // the stacked system over M n constants: R = min1(A + B R)
                    const int32_t N = M * n;
                    const size_t NN = static_cast<size_t>(N) * N;
                    uint8_t *Bs = pool.alloc(NN), *As = pool.alloc(NN), *Sb = pool.alloc(NN);
                    auto *bits = static_cast<uint64_t *>(ws.get("pg_sbits", static_cast<size_t>(N) * ((N + 63) / 64) * 8));
                    if (!Bs || !As || !Sb || !bits) {
                        set_error("program: device allocation failed (stacked system of %d x %d)", N, N);
                        return DL_ENOMEM;
                    }
                    // B = [B_hj] (M x M blocks), A = [A_h] in block column 0; R_h is block (h, 0)
                    PCK(cudaMemsetAsync(Bs, 0, NN, s));
                    PCK(cudaMemsetAsync(As, 0, NN, s));
                    for (int h = 0; h < M; ++h) {
                        PCK(cudaMemcpy2DAsync(As + static_cast<size_t>(h) * n * N, N, Aa[h], n, n, n,
                                              cudaMemcpyDeviceToDevice, s));
                        for (int j = 0; j < M; ++j)
                            if (Bj[h][j])
                                PCK(cudaMemcpy2DAsync(Bs + static_cast<size_t>(h) * n * N + static_cast<size_t>(j) * n,
                                                      N, Bj[h][j], n, n, n, cudaMemcpyDeviceToDevice, s));
                    }
                    if ((rc = tail(N, Bs, As, bits))) return rc;
                    PCK(unpack_bits_u8(bits, N, Sb, ws.status, s));
                    ++R.launches;
                    for (int h = 0; h < M; ++h) {
                        if ((rc = R.mat(&out[h]))) return rc;
                        PCK(cudaMemcpy2DAsync(out[h], n, Sb + static_cast<size_t>(h) * n * N, N, n, n,
                                              cudaMemcpyDeviceToDevice, s));
                    }
                }
                if (!left)
                    for (int h = 0; h < M; ++h)
                        if ((rc = R.transpose(out[h], &out[h]))) return rc;
                how = std::string(left ? "tail recursive (Sec. 6.1)" : "tail recursive on the transposes (Sec. 6.1)") +
                      (M == 1 ? ": R = min1(A + B0 R)" : ": mutually recursive, one closure of the stacked system");
            } else if (trans_left || trans_right) {
                // R = A + B R^T gives R = min1(A + B A^T + B R B^T); R = A + R^T C gives
                // R = min1(A + A^T C + C^T R C)  (the two-sided reduction of eq. matrixeq:trans:2)
                uint8_t *sum = nullptr, *at = nullptr, *rhs = nullptr, *P = nullptr;
                if ((rc = coeff_sum(trans_left, &sum)) || (rc = R.transpose(A[0], &at))) return rc;
                if (trans_left) {
                    P = sum;
                    if ((rc = R.product(sum, at, &rhs))) return rc;
                } else {
                    if ((rc = R.transpose(sum, &P)) || (rc = R.product(at, sum, &rhs))) return rc;
                }
                if ((rc = R.or_into(rhs, A[0]))) return rc;
                if ((rc = R.two_sided(P, rhs, &out[0]))) return rc;
                how = "transposed class (Sec. 6.2) through the two-sided reduction, same-generation solver";
            } else if (sg_form) {
                if ((rc = R.two_sided(terms[0][0].B, A[0], &out[0]))) return rc;
                how = "two-sided class (Sec. 6.3) in the same-generation form R = min1(A + P R P^T)";
            } else {
                // the series of Lemma 3 from 0 until nothing changes; each iteration's
                // temporaries live in a pool of their own
                std::vector<uint8_t *> cur(M, nullptr), nxt(M, nullptr);
                for (int h = 0; h < M; ++h)
                    if ((rc = R.zero(&cur[h])) || (rc = R.mat(&nxt[h]))) return rc;
                const int64_t cap = static_cast<int64_t>(M) * n * n + 2;
                int64_t it = 0;
                for (bool settled = false; !settled; ++it) {
                    if (it > cap) {
                        set_error("program: the series of layer %zu did not settle", l);
                        return DL_ENOTCONV;
                    }
                    {
                        Pool inner;
                        R.pool = &inner;
                        for (int h = 0; h < M && !rc; ++h) {
                            if ((rc = R.copy(nxt[h], A[h]))) break;
                            for (const Term &t : terms[h]) {
                                uint8_t *rj = cur[t.j], *x = nullptr, *y = nullptr;
                                if (t.transposed && (rc = R.transpose(rj, &rj))) break;
                                if ((rc = R.product(t.B, rj, &x)) || (rc = R.product(x, t.C, &y))) break;
                                if ((rc = R.or_into(nxt[h], y))) break;
                            }
                        }
                        settled = true;
                        for (int h = 0; h < M && settled && !rc; ++h) rc = R.equal(nxt[h], cur[h], &settled);
                        R.pool = &pool;
                        if (rc) return rc;
                    }
                    std::swap(cur, nxt);
                }
                out = cur;
                how = "the series of Lemma 3 (eq. series:gen) on FP8 products, " + std::to_string(it) + " iterations";
            }
        }
        plan << "layer " << l << ": {";
        for (int h = 0; h < M; ++h) plan << (h ? ", " : "") << preds[h];
        plan << "} " << how << "\n";
        for (int h = 0; h < M; ++h) model[preds[h]] = out[h];
    }
    // keep the models (program-owned copies)
    for (auto &kv : model) {
        uint8_t *&d = p->rel[kv.first];
        if (!d && device_alloc(reinterpret_cast<void **>(&d), nbytes) != cudaSuccess) {
            cudaGetLastError();
            p->rel.erase(kv.first);
            set_error("program: device allocation failed");
            return DL_ENOMEM;
        }
        if (n > 0) PCK(cudaMemcpyAsync(d, kv.second, static_cast<size_t>(n) * n, cudaMemcpyDeviceToDevice, s));
    }
    PCK(cudaStreamSynchronize(s));
    p->plan = plan.str();
    p->ran = true;
    if (st) {
        st->gemm_launches = R.gemms;
        st->gpu_launches = R.launches;
        st->ms_total = R.ms;
        st->iters = static_cast<int32_t>(p->layers.size());
    }
    return DL_OK;
}

dl_status program_get(dl_program *p, Workspace &ws, cudaStream_t s, const char *pred, uint64_t *out_bits, dl_mem mem) {
    if (!p->ran || !p->idb.count(pred)) {
        set_error(p->ran ? "program: %s is not a predicate defined by the program" : "program: run it first (%s)", pred);
        return DL_EINVAL;
    }
    const int32_t n = p->n;
    if (n == 0) return DL_OK;
    const int64_t np = (static_cast<int64_t>(n) + 255) / 256 * 256, wp = np / 64, w = (n + 63) / 64;
    auto *M = static_cast<uint64_t *>(ws.get("pg_out", static_cast<size_t>(np) * wp * 8));
    if (!M) {
        set_error("program: device allocation failed");
        return DL_ENOMEM;
    }
    PCK(pack_bits(p->rel[pred], n, static_cast<int>(np), wp, M, ws.status, s));
    PCK(cudaMemcpy2DAsync(out_bits, w * 8, M, wp * 8, w * 8, n,
                          mem == DL_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    PCK(cudaStreamSynchronize(s));
    return DL_OK;
}

std::string program_describe(const dl_program *p) {
    std::ostringstream o;
    o << "base:";
    for (const std::string &e : p->edb) o << " " << e;
    o << "\ndefined:";
    for (const std::string &r : p->idb) o << " " << r;
    o << "\n";
    for (size_t l = 0; l < p->layers.size(); ++l) {
        o << "layer " << l << ":";
        for (const std::string &r : p->layers[l]) o << " " << r;
        o << "\n";
    }
    if (p->ran) o << "plan:\n" << p->plan;
    return o.str();
}

dl_ctx *program_ctx(const dl_program *p) { return p->ctx; }

}  // namespace dl
