// extern "C" entry points declared in include/ckks_mulk.h: argument checks,
// tuple -> view marshalling, error codes. No exception crosses the ABI.
#include <cmath>
#include <cstring>
#include <new>

#include "../../include/ckks_mulk.h"
#include "engine.h"
#include "internal.h"
#include "plan.h"
#include "rns.h"

using namespace ckks;


static long long evk_words(const Context &C, uint32_t t_max) {
    return (long long)(t_max - 1) * C.dnum * 2 * (C.L + C.K) * C.N;
}

// checksum of the set's key buffer (synchronous on `st`)
static cudaError_t evk_checksum(const Context &C, const u64 *keys, uint32_t t_max, cudaStream_t st,
                                unsigned long long &sum) {
    cudaError_t e = cudaMemsetAsync(C.d_check + 1, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = launch_checksum(C, keys, evk_words(C, t_max), C.d_check + 1, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&sum, C.d_check + 1, sizeof(sum), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
}

// reads and clears the residue-check counter (synchronous on `st`)
static cudaError_t take_residue_count(const Context &C, cudaStream_t st, unsigned long long &bad) {
    cudaError_t e = cudaMemcpyAsync(&bad, C.d_check, sizeof(bad), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(C.d_check, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
}

static int cuda_fail(ckks_context *ctx, cudaError_t e) {
    if (e != cudaSuccess) {
        ctx->c.sticky.store((int)e);
        return CKKS_ECUDA;
    }
    return CKKS_OK;
}

static int finish(ckks_context *ctx, int rc, cudaError_t e) {
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    return rc;
}

static bool tuple_ok(const ckks_tuple *t, uint32_t L) {
    return t && t->data && t->level >= 1 && t->level <= L && t->poly_stride >= t->level && t->n_polys >= 1 &&
           t->n_polys <= CKKS_MAX_TUPLE;
}

static LimbView tview(const ckks_tuple &t, int N, i64 bstride = 0) {
    LimbView v;
    v.ptr = (u64 *)t.data;
    v.bstride = bstride;
    v.pstride = (i64)t.poly_stride * N;
    return v;
}

static cudaStream_t S(void *s) { return (cudaStream_t)s; }

extern "C" {

int ckks_context_create(const ckks_params *params, int device, ckks_context **out) {
    if (!params || !out || !params->q || !params->p) return CKKS_EINVAL;
    *out = nullptr;
    ckks_context *ctx = new (std::nothrow) ckks_context();
    if (!ctx) return CKKS_ENOMEM;
    int rc = context_build(ctx->c, params->log_n, params->L, params->K, params->dnum, (const u64 *)params->q,
                           (const u64 *)params->p, device);
    if (rc != 0) {
        context_release(ctx->c);
        delete ctx;
        return rc == -5 ? CKKS_ECUDA : CKKS_EINVAL;
    }
    *out = ctx;
    return CKKS_OK;
}

void ckks_context_destroy(ckks_context *ctx) {
    if (!ctx) return;
    context_release(ctx->c);
    delete ctx;
}

int ckks_keygen_workspace_size(const ckks_context *ctx, size_t *bytes) {
    if (!ctx || !bytes) return CKKS_EINVAL;
    *bytes = (size_t)3 * (ctx->c.L + ctx->c.K) * ctx->c.N * sizeof(u64);
    return CKKS_OK;
}

int ckks_keygen_evk(ckks_context *ctx, uint32_t t_max, const int64_t *s, const uint64_t *a, const int64_t *e,
                    uint64_t *keys, void *workspace, size_t ws_bytes, void *stream) {
    if (!ctx || !s || !a || !e || !keys || !workspace || t_max < 2 || t_max > 13) return CKKS_EINVAL;
    const Context &C = ctx->c;
    size_t need;
    ckks_keygen_workspace_size(ctx, &need);
    if (ws_bytes < need) return CKKS_ENOMEM;
    cudaSetDevice(C.device);
    const int NP = C.L + C.K;
    const size_t plane = (size_t)NP * C.N;
    u64 *Sb = (u64 *)workspace, *St = Sb + plane, *E = St + plane;
    cudaStream_t st = S(stream);
    LimbView v = {Sb, 0, (i64)plane};
    cudaError_t err = launch_signed_to_res(C, (const long long *)s, Sb, st);
    if (err == cudaSuccess) {
        LimbJobs J;
        memset(&J, 0, sizeof(J));
        J.n_batch = 1;
        J.n_polys = 1;
        J.n_limbs = NP;
        for (int i = 0; i < NP; ++i) J.slot[i] = J.dslot[i] = J.prime[i] = (uint8_t)i;
        LoadSpec L{};
        L.mode = LD_PLAIN;
        L.a = v;
        StoreSpec Sp{};
        Sp.mode = ST_REDUCE;
        Sp.dst = v;
        err = ntt_transform(C, true, J, L, Sp, nullptr, st);
        if (err == cudaSuccess) err = cudaMemcpyAsync(St, Sb, plane * sizeof(u64), cudaMemcpyDeviceToDevice, st);
        for (uint32_t t = 2; t <= t_max && err == cudaSuccess; ++t) {
            err = launch_pointwise_mul(C, St, Sb, st);
            for (int b = 0; b < C.dnum && err == cudaSuccess; ++b) {
                const size_t kb = (size_t)(t - 2) * C.dnum + b;
                err = launch_signed_to_res(C, (const long long *)(e + kb * C.N), E, st);
                if (err != cudaSuccess) break;
                LoadSpec Le{};
                Le.mode = LD_PLAIN;
                Le.a = LimbView{E, 0, (i64)plane};
                StoreSpec Se{};
                Se.mode = ST_REDUCE;
                Se.dst = Le.a;
                err = ntt_transform(C, true, J, Le, Se, nullptr, st);
                if (err != cudaSuccess) break;
                err = launch_keygen(C, Sb, St, E, (const u64 *)a + kb * plane, (u64 *)keys + kb * 2 * plane, b, st);
            }
        }
    }
    return finish(ctx, CKKS_OK, err);
}

int ckks_evk_set_create(ckks_context *ctx, uint32_t t_max, uint64_t *keys, void *stream, ckks_evk_set **out) {
    if (!out) return CKKS_EINVAL;
    *out = nullptr;
    // the key MAC reads keys with 16-byte loads
    if (!ctx || !keys || t_max < 2 || t_max > 13 || (uintptr_t)keys % 16) return CKKS_EINVAL;
    const Context &C = ctx->c;
    cudaSetDevice(C.device);
    long long rows = (long long)(t_max - 1) * C.dnum * 2 * (C.L + C.K);
    cudaError_t err = launch_keyprep(C, (u64 *)keys, rows, S(stream));
    if (err != cudaSuccess) return cuda_fail(ctx, err);
    unsigned long long sum = 0;
    err = evk_checksum(C, (const u64 *)keys, t_max, S(stream), sum);
    if (err != cudaSuccess) return cuda_fail(ctx, err);
    ckks_evk_set *set = new (std::nothrow) ckks_evk_set{ctx, (u64 *)keys, t_max, sum};
    if (!set) return CKKS_ENOMEM;
    *out = set;
    return CKKS_OK;
}

void ckks_evk_set_destroy(ckks_evk_set *set) { delete set; }

int ckks_evk_verify(ckks_evk_set *set, void *stream) {
    if (!set || !set->ctx) return CKKS_EINVAL;
    const Context &C = set->ctx->c;
    cudaSetDevice(C.device);
    unsigned long long sum = 0;
    cudaError_t err = evk_checksum(C, set->keys, set->t_max, S(stream), sum);
    if (err != cudaSuccess) return cuda_fail(set->ctx, err);
    return sum == set->sum ? CKKS_OK : CKKS_ECHECK;
}

int ckks_check_residues(ckks_context *ctx, const ckks_tuple *t, uint64_t *bad, void *stream) {
    if (!ctx || !t || !bad || !tuple_ok(t, ctx->c.L)) return CKKS_EINVAL;
    const Context &C = ctx->c;
    cudaSetDevice(C.device);
    cudaStream_t st = S(stream);
    unsigned long long n = 0;
    cudaError_t err = cudaMemsetAsync(C.d_check, 0, sizeof(unsigned long long), st);
    if (err == cudaSuccess) err = launch_range_check(C, tview(*t, C.N), 1, (int)t->n_polys, (int)t->level, st);
    if (err == cudaSuccess) err = take_residue_count(C, st, n);
    if (err != cudaSuccess) return cuda_fail(ctx, err);
    *bad = n;
    return CKKS_OK;
}

int ckks_plan_create(ckks_context *ctx, uint32_t k, const char *partition, ckks_plan **out) {
    (void)ctx;
    if (!out) return CKKS_EINVAL;
    *out = nullptr;
    ckks_plan *p = new (std::nothrow) ckks_plan();
    if (!p) return CKKS_ENOMEM;
    if (plan_build(p->p, (int)k, partition) != 0) {
        delete p;
        return CKKS_EINVAL;
    }
    *out = p;
    return CKKS_OK;
}

void ckks_plan_destroy(ckks_plan *plan) { delete plan; }

int ckks_plan_describe(const ckks_plan *plan, uint32_t *depth, uint32_t *rs_units, uint32_t *n_nodes) {
    if (!plan) return CKKS_EINVAL;
    if (depth) *depth = (uint32_t)plan->p.depth;
    if (rs_units) *rs_units = (uint32_t)plan->p.rs_units;
    if (n_nodes) *n_nodes = (uint32_t)plan->p.nodes.size();
    return CKKS_OK;
}

int ckks_plan_optimize(uint32_t k, int criterion, uint32_t level, uint32_t K, uint32_t alpha, char *text,
                       size_t text_len, double *cost) {
    if (!text || text_len == 0 || criterion < 0 || criterion > 2 || (criterion >= 1 && alpha == 0))
        return CKKS_EINVAL;
    std::string best;
    double c = 0;
    int rc = plan_optimize((int)k, criterion, (int)level, (int)K, (int)alpha, best, c);
    if (rc == -2) return CKKS_ELEVEL;
    if (rc != 0 || best.size() + 1 > text_len) return CKKS_EINVAL;
    memcpy(text, best.c_str(), best.size() + 1);
    if (cost) *cost = c;
    return CKKS_OK;
}

int ckks_plan_cost(const ckks_plan *plan, int criterion, uint32_t level, uint32_t K, uint32_t alpha, double *cost) {
    if (!plan || !cost || criterion < 0 || criterion > 2 || (criterion >= 1 && alpha == 0)) return CKKS_EINVAL;
    if (criterion >= 1 && (int)level <= plan->p.depth) return CKKS_ELEVEL;
    *cost = plan_cost(plan->p, criterion, (int)level, (int)K, (int)alpha);
    return CKKS_OK;
}

int ckks_workspace_size(const ckks_context *ctx, const ckks_plan *plan, uint32_t level, uint32_t batch,
                        size_t *bytes) {
    if (!ctx || !plan || !bytes || batch < 1) return CKKS_EINVAL;
    if (level > (uint32_t)ctx->c.L || (int)level <= plan->p.depth) return CKKS_ELEVEL;
    *bytes = mul_k_ws_bytes(ctx->c, plan->p, (int)level, (int)batch);
    return CKKS_OK;
}

// scale of the result: product of input scales / primes divided at each node

static int mul_k_common(ckks_context *ctx, const ckks_tuple *ct, uint32_t k, uint32_t batch, const ckks_evk_set *evk,
                        const ckks_plan *plan, ckks_tuple *out, void *ws, size_t ws_bytes, void *stream) {
    if (!ctx || !ct || !evk || !plan || !out || batch < 1) return CKKS_EINVAL;
    const Context &C = ctx->c;
    const Plan &P = plan->p;
    if ((int)k != P.k || evk->ctx != ctx) return CKKS_EINVAL;
    const uint32_t level = ct[0].level;
    for (uint32_t i = 0; i < k * batch; ++i) {
        const ckks_tuple &t = ct[i];
        if (!tuple_ok(&t, C.L) || t.n_polys != 2 || t.ntt_form != 1 || t.level != level ||
            t.poly_stride != ct[i % k].poly_stride)
            return CKKS_EINVAL;
    }
    if ((int)level <= P.depth) return CKKS_ELEVEL;
    if (evk->t_max < k) return CKKS_EKEY;
    const uint32_t out_level = level - P.depth;
    std::vector<LimbView> in(k);
    for (uint32_t u = 0; u < k; ++u) {
        i64 bs = 0;
        if (batch > 1) bs = (i64)(ct[k + u].data - ct[u].data);
        for (uint32_t b = 0; b < batch; ++b)
            if (ct[b * k + u].data != ct[u].data + b * bs) return CKKS_EINVAL;
        in[u] = tview(ct[u], C.N, bs);
    }
    for (uint32_t b = 0; b < batch; ++b) {
        if (!out[b].data) return CKKS_EINVAL;
        if (out[b].poly_stride == 0) out[b].poly_stride = out_level;
        if (out[b].poly_stride < out_level || out[b].poly_stride != out[0].poly_stride) return CKKS_EINVAL;
    }
    i64 obs = batch > 1 ? (i64)(out[1].data - out[0].data) : 0;
    if (batch > 1 && obs == 0) return CKKS_EINVAL;  // batch elements would write one output
    for (uint32_t b = 0; b < batch; ++b)
        if (out[b].data != out[0].data + b * obs) return CKKS_EINVAL;
    size_t need = mul_k_ws_bytes(C, P, (int)level, (int)batch);
    if (!ws || ws_bytes < need) return CKKS_ENOMEM;
    cudaSetDevice(C.device);
    cudaError_t err;
    int rc = run_mul_k_ws(C, P, (int)level, (int)batch, in.data(), tview(out[0], C.N, obs), evk->keys,
                          (int)evk->t_max, ws, ws_bytes, S(stream), err);
    if (rc == -3) return CKKS_EKEY;
    if (err != cudaSuccess || rc != 0) return cuda_fail(ctx, err == cudaSuccess ? cudaErrorUnknown : err);
    if (C.tune_check_residues) {
        unsigned long long bad = 0;
        err = take_residue_count(C, S(stream), bad);
        if (err != cudaSuccess) return cuda_fail(ctx, err);
        if (bad) return CKKS_ECHECK;
    }
    for (uint32_t b = 0; b < batch; ++b) {
        std::vector<double> sc(k);
        for (uint32_t u = 0; u < k; ++u) sc[u] = ct[b * k + u].scale;
        out[b].n_polys = 2;
        out[b].level = out_level;
        out[b].ntt_form = 1;
        out[b].scale = plan_scale(C, P, (int)level, sc.data());
    }
    return CKKS_OK;
}

int ckks_mul_k(ckks_context *ctx, const ckks_tuple *ct, uint32_t k, const ckks_evk_set *evk, const ckks_plan *plan,
               ckks_tuple *out, void *workspace, size_t ws_bytes, void *stream) {
    return mul_k_common(ctx, ct, k, 1, evk, plan, out, workspace, ws_bytes, stream);
}

int ckks_mul_k_batch(ckks_context *ctx, const ckks_tuple *ct, uint32_t k, uint32_t batch, const ckks_evk_set *evk,
                     const ckks_plan *plan, ckks_tuple *out, void *workspace, size_t ws_bytes, void *stream) {
    return mul_k_common(ctx, ct, k, batch, evk, plan, out, workspace, ws_bytes, stream);
}

int ckks_requests_workspace_size(const ckks_context *ctx, const ckks_request *req, uint32_t n, size_t *bytes) {
    if (!ctx || !req || !bytes || n < 1) return CKKS_EINVAL;
    size_t need = 0;
    for (uint32_t i = 0; i < n; ++i) {
        const ckks_request &r = req[i];
        if (!r.ct || !r.plan || r.batch < 1 || (int)r.k != r.plan->p.k) return CKKS_EINVAL;
        const uint32_t level = r.ct[0].level;
        if (level <= (uint32_t)r.plan->p.depth || level > (uint32_t)ctx->c.L) return CKKS_ELEVEL;
        need = std::max(need, mul_k_ws_bytes(ctx->c, r.plan->p, (int)level, (int)r.batch));
    }
    *bytes = need;
    return CKKS_OK;
}

int ckks_mul_k_requests(ckks_context *ctx, const ckks_request *req, uint32_t n, uint32_t *done, void *workspace,
                        size_t ws_bytes, void *stream) {
    if (done) *done = 0;
    if (!ctx || !req || n < 1) return CKKS_EINVAL;
    for (uint32_t i = 0; i < n; ++i) {
        const ckks_request &r = req[i];
        const int rc = mul_k_common(ctx, r.ct, r.k, r.batch, r.evk, r.plan, r.out, workspace, ws_bytes, stream);
        if (rc != CKKS_OK) return rc;
        if (done) *done = i + 1;
    }
    return CKKS_OK;
}

// batch stride of a [batch] tuple array; -1 if the pointers are not evenly spaced
static i64 batch_stride(const ckks_tuple *t, uint32_t batch) {
    i64 bs = batch > 1 ? (i64)(t[1].data - t[0].data) : 0;
    for (uint32_t b = 0; b < batch; ++b)
        if (t[b].data != t[0].data + b * bs) return -1;
    return bs;
}

int ckks_mul2_workspace_size(const ckks_context *ctx, uint32_t level, uint32_t batch, size_t *bytes) {
    if (!ctx || !bytes || batch < 1) return CKKS_EINVAL;
    if (level < 2 || level > (uint32_t)ctx->c.L) return CKKS_ELEVEL;
    *bytes = mul2_ws_bytes(ctx->c, (int)level, (int)batch);
    return CKKS_OK;
}

int ckks_mul2_batch(ckks_context *ctx, const ckks_tuple *a, const ckks_tuple *b, uint32_t batch,
                    const ckks_evk_set *evk, ckks_tuple *out, void *workspace, size_t ws_bytes, void *stream) {
    if (!ctx || !a || !b || !evk || !out || evk->ctx != ctx || batch < 1) return CKKS_EINVAL;
    const Context &C = ctx->c;
    for (uint32_t i = 0; i < batch; ++i) {
        if (!tuple_ok(&a[i], C.L) || !tuple_ok(&b[i], C.L) || a[i].n_polys != 2 || b[i].n_polys != 2 ||
            !a[i].ntt_form || !b[i].ntt_form || !out[i].data || a[i].level != a[0].level ||
            b[i].level != b[0].level || a[i].poly_stride != a[0].poly_stride ||
            b[i].poly_stride != b[0].poly_stride)
            return CKKS_EINVAL;
    }
    const int level = (int)std::min(a[0].level, b[0].level);
    if (level < 2) return CKKS_ELEVEL;
    if (evk->t_max < 2) return CKKS_EKEY;
    for (uint32_t i = 0; i < batch; ++i) {
        if (out[i].poly_stride == 0) out[i].poly_stride = level - 1;
        if ((int)out[i].poly_stride < level - 1 || out[i].poly_stride != out[0].poly_stride) return CKKS_EINVAL;
    }
    i64 as = batch_stride(a, batch), bs = batch_stride(b, batch), os = batch_stride(out, batch);
    if (as < 0 || bs < 0 || os < 0 || (batch > 1 && os == 0)) return CKKS_EINVAL;
    size_t need = mul2_ws_bytes(C, level, (int)batch);
    if (!workspace || ws_bytes < need) return CKKS_ENOMEM;
    cudaSetDevice(C.device);
    cudaError_t err;
    int rc = run_mul2_ws(C, level, (int)batch, tview(a[0], C.N, as), tview(b[0], C.N, bs), tview(out[0], C.N, os),
                         evk->keys, workspace, ws_bytes, S(stream), err);
    if (err != cudaSuccess || rc != 0) return cuda_fail(ctx, err == cudaSuccess ? cudaErrorUnknown : err);
    for (uint32_t i = 0; i < batch; ++i) {
        out[i].n_polys = 2;
        out[i].level = level - 1;
        out[i].ntt_form = 1;
        out[i].scale = a[i].scale * b[i].scale / (double)C.primes[level - 1];
    }
    return CKKS_OK;
}

int ckks_mul2(ckks_context *ctx, const ckks_tuple *a, const ckks_tuple *b, const ckks_evk_set *evk, ckks_tuple *out,
              void *workspace, size_t ws_bytes, void *stream) {
    return ckks_mul2_batch(ctx, a, b, 1, evk, out, workspace, ws_bytes, stream);
}

int ckks_tensor(ckks_context *ctx, const ckks_tuple *in, uint32_t m, ckks_tuple *out, void *stream) {
    if (!ctx || !in || !out || !out->data || m < 1 || m > CKKS_MAX_CHILDREN) return CKKS_EINVAL;
    const Context &C = ctx->c;
    uint32_t level = 1u << 30, np = 1;
    std::vector<LimbView> v(m);
    std::vector<int> polys(m);
    double scale = 1.0;
    for (uint32_t i = 0; i < m; ++i) {
        if (!tuple_ok(&in[i], C.L) || !in[i].ntt_form) return CKKS_EINVAL;
        level = std::min(level, in[i].level);
        np += in[i].n_polys - 1;
        v[i] = tview(in[i], C.N);
        polys[i] = (int)in[i].n_polys;
        scale *= in[i].scale;
    }
    if (np > CKKS_MAX_TUPLE) return CKKS_EINVAL;
    if (out->poly_stride == 0) out->poly_stride = level;
    if (out->poly_stride < level) return CKKS_EINVAL;
    cudaSetDevice(C.device);
    cudaError_t err = run_tensor(C, 1, (int)level, (int)m, v.data(), polys.data(), tview(*out, C.N), S(stream));
    if (err != cudaSuccess) return cuda_fail(ctx, err);
    out->n_polys = np;
    out->level = level;
    out->ntt_form = 1;
    out->scale = scale;
    return CKKS_OK;
}

int ckks_relin_workspace_size(const ckks_context *ctx, uint32_t n, uint32_t level, size_t *bytes) {
    if (!ctx || !bytes || n < 2 || level < 1 || level > (uint32_t)ctx->c.L) return CKKS_EINVAL;
    *bytes = relin_ws_bytes(ctx->c, (int)n, (int)level, 1);
    return CKKS_OK;
}

int ckks_relin(ckks_context *ctx, const ckks_tuple *d, const ckks_evk_set *evk, uint32_t out_ntt, ckks_tuple *out,
               void *workspace, size_t ws_bytes, void *stream) {
    if (!ctx || !d || !evk || !out || !out->data || evk->ctx != ctx) return CKKS_EINVAL;
    const Context &C = ctx->c;
    if (!tuple_ok(d, C.L) || d->n_polys < 3 || !d->ntt_form) return CKKS_EINVAL;
    const uint32_t n = d->n_polys - 1;
    if (evk->t_max < n) return CKKS_EKEY;
    if (out->poly_stride == 0) out->poly_stride = d->level;
    if (out->poly_stride < d->level) return CKKS_EINVAL;
    size_t need = relin_ws_bytes(C, (int)n, (int)d->level, 1);
    if (!workspace || ws_bytes < need) return CKKS_ENOMEM;
    cudaSetDevice(C.device);
    cudaError_t err;
    int rc = run_relin_ws(C, 1, (int)n, (int)d->level, tview(*d, C.N), evk->keys, out_ntt != 0, tview(*out, C.N),
                          workspace, ws_bytes, S(stream), err);
    if (err != cudaSuccess || rc != 0) return cuda_fail(ctx, err == cudaSuccess ? cudaErrorUnknown : err);
    out->n_polys = 2;
    out->level = d->level;
    out->ntt_form = out_ntt ? 1 : 0;
    out->scale = d->scale;
    return CKKS_OK;
}

// ---------------------------------------------------------------------------
// Galois automorphisms and rotation
// ---------------------------------------------------------------------------
static bool galois_ok(const Context &C, uint32_t g) { return (g & 1u) && g < (uint32_t)(2 * C.N); }

int ckks_galois_element(const ckks_context *ctx, int32_t r, uint32_t *g) {
    if (!ctx || !g) return CKKS_EINVAL;
    const Context &C = ctx->c;
    if (C.N < 4) return CKKS_EINVAL;
    const uint64_t M = 2ull * (uint64_t)C.N, half = (uint64_t)C.N / 2;  // 5 has order N/2 mod 2N
    uint64_t e = (uint64_t)(((int64_t)r % (int64_t)half + (int64_t)half) % (int64_t)half);
    uint64_t x = 1, b = 5 % M;
    for (; e; e >>= 1, b = b * b % M)
        if (e & 1) x = x * b % M;
    *g = (uint32_t)x;
    return CKKS_OK;
}

int ckks_automorphism(ckks_context *ctx, const ckks_tuple *in, uint32_t g, ckks_tuple *out, void *stream) {
    if (!ctx || !in || !out || !out->data) return CKKS_EINVAL;
    const Context &C = ctx->c;
    if (!tuple_ok(in, C.L) || !in->ntt_form || !galois_ok(C, g) || out->data == in->data) return CKKS_EINVAL;
    if (out->poly_stride == 0) out->poly_stride = in->level;
    if (out->poly_stride < in->level) return CKKS_EINVAL;
    AutoMap map{};
    map.n_out = (int)in->n_polys;
    for (int p = 0; p < map.n_out; ++p) map.src[p] = p;
    cudaSetDevice(C.device);
    cudaError_t err = launch_automorphism(C, tview(*in, C.N), tview(*out, C.N), map, 1, (int)in->level, g, S(stream));
    if (err != cudaSuccess) return cuda_fail(ctx, err);
    out->n_polys = in->n_polys;
    out->level = in->level;
    out->ntt_form = 1;
    out->scale = in->scale;
    return CKKS_OK;
}

int ckks_keygen_galois(ckks_context *ctx, uint32_t g, const int64_t *s, const uint64_t *a, const int64_t *e,
                       uint64_t *keys, void *workspace, size_t ws_bytes, void *stream) {
    if (!ctx || !s || !a || !e || !keys || !workspace) return CKKS_EINVAL;
    const Context &C = ctx->c;
    if (!galois_ok(C, g)) return CKKS_EINVAL;
    size_t need;
    ckks_keygen_workspace_size(ctx, &need);
    if (ws_bytes < need) return CKKS_ENOMEM;
    cudaSetDevice(C.device);
    const int NP = C.L + C.K;
    const size_t plane = (size_t)NP * C.N;
    u64 *Sb = (u64 *)workspace, *Sg = Sb + plane, *E = Sg + plane;
    cudaStream_t st = S(stream);
    LimbJobs J;
    memset(&J, 0, sizeof(J));
    J.n_batch = 1;
    J.n_polys = 1;
    J.n_limbs = NP;
    for (int i = 0; i < NP; ++i) J.slot[i] = J.dslot[i] = J.prime[i] = (uint8_t)i;
    auto ntt_plane = [&](u64 *buf) {
        LoadSpec L{};
        L.mode = LD_PLAIN;
        L.a = LimbView{buf, 0, (i64)plane};
        StoreSpec Sp{};
        Sp.mode = ST_REDUCE;
        Sp.dst = L.a;
        return ntt_transform(C, true, J, L, Sp, nullptr, st);
    };
    // S = NTT(s), S_g = sigma_g(S) (a permutation in the NTT domain)
    cudaError_t err = launch_signed_to_res(C, (const long long *)s, Sb, st);
    if (err == cudaSuccess) err = ntt_plane(Sb);
    if (err == cudaSuccess) {
        AutoMap map{};
        map.n_out = 1;
        map.src[0] = 0;
        err = launch_automorphism(C, LimbView{Sb, 0, (i64)plane}, LimbView{Sg, 0, (i64)plane}, map, 1, NP, g, st);
    }
    for (int b = 0; b < C.dnum && err == cudaSuccess; ++b) {
        err = launch_signed_to_res(C, (const long long *)(e + (size_t)b * C.N), E, st);
        if (err == cudaSuccess) err = ntt_plane(E);
        if (err == cudaSuccess)
            err = launch_keygen(C, Sb, Sg, E, (const u64 *)a + b * plane, (u64 *)keys + (size_t)b * 2 * plane, b, st);
    }
    if (err != cudaSuccess) return cuda_fail(ctx, err);
    return CKKS_OK;
}

int ckks_rotate_workspace_size(const ckks_context *ctx, uint32_t level, uint32_t batch, size_t *bytes) {
    if (!ctx || !bytes || batch < 1) return CKKS_EINVAL;
    if (level < 1 || level > (uint32_t)ctx->c.L) return CKKS_ELEVEL;
    *bytes = rotate_ws_bytes(ctx->c, (int)level, (int)batch);
    return CKKS_OK;
}

int ckks_rotate_batch(ckks_context *ctx, const ckks_tuple *in, uint32_t batch, uint32_t g, const ckks_evk_set *gk,
                      ckks_tuple *out, void *workspace, size_t ws_bytes, void *stream) {
    if (!ctx || !in || !gk || !out || gk->ctx != ctx || batch < 1) return CKKS_EINVAL;
    const Context &C = ctx->c;
    if (!galois_ok(C, g)) return CKKS_EINVAL;
    for (uint32_t i = 0; i < batch; ++i) {
        if (!tuple_ok(&in[i], C.L) || in[i].n_polys != 2 || !in[i].ntt_form || !out[i].data ||
            in[i].level != in[0].level || in[i].poly_stride != in[0].poly_stride)
            return CKKS_EINVAL;
    }
    const int level = (int)in[0].level;
    for (uint32_t i = 0; i < batch; ++i) {
        if (out[i].poly_stride == 0) out[i].poly_stride = in[i].data == out[i].data ? in[i].poly_stride : level;
        if ((int)out[i].poly_stride < level || out[i].poly_stride != out[0].poly_stride) return CKKS_EINVAL;
    }
    i64 is = batch_stride(in, batch), os = batch_stride(out, batch);
    if (is < 0 || os < 0 || (batch > 1 && os == 0)) return CKKS_EINVAL;
    size_t need = rotate_ws_bytes(C, level, (int)batch);
    if (!workspace || ws_bytes < need) return CKKS_ENOMEM;
    cudaSetDevice(C.device);
    cudaError_t err;
    int rc = run_rotate_ws(C, (int)batch, level, g, tview(in[0], C.N, is), tview(out[0], C.N, os), gk->keys,
                           workspace, ws_bytes, S(stream), err);
    if (err != cudaSuccess || rc != 0) return cuda_fail(ctx, err == cudaSuccess ? cudaErrorUnknown : err);
    for (uint32_t i = 0; i < batch; ++i) {
        out[i].n_polys = 2;
        out[i].level = (uint32_t)level;
        out[i].ntt_form = 1;
        out[i].scale = in[i].scale;
    }
    return CKKS_OK;
}

int ckks_rotate(ckks_context *ctx, const ckks_tuple *in, uint32_t g, const ckks_evk_set *gk, ckks_tuple *out,
                void *workspace, size_t ws_bytes, void *stream) {
    return ckks_rotate_batch(ctx, in, 1, g, gk, out, workspace, ws_bytes, stream);
}

int ckks_rescale_workspace_size(const ckks_context *ctx, uint32_t n_polys, uint32_t level, uint32_t mu,
                                size_t *bytes) {
    if (!ctx || !bytes || mu < 1 || mu >= level || level > (uint32_t)ctx->c.L || n_polys < 1) return CKKS_EINVAL;
    *bytes = rescale_ws_bytes(ctx->c, (int)n_polys, (int)level, (int)mu, 1);
    return CKKS_OK;
}

int ckks_rescale_multi(ckks_context *ctx, const ckks_tuple *in, uint32_t mu, ckks_tuple *out, void *workspace,
                       size_t ws_bytes, void *stream) {
    if (!ctx || !in || !out || !out->data) return CKKS_EINVAL;
    const Context &C = ctx->c;
    if (!tuple_ok(in, C.L) || !in->ntt_form) return CKKS_EINVAL;
    if (mu < 1 || mu >= in->level) return CKKS_ELEVEL;
    const uint32_t ol = in->level - mu;
    if (out->poly_stride == 0) out->poly_stride = out->data == in->data ? in->poly_stride : ol;
    if (out->poly_stride < ol) return CKKS_EINVAL;
    if (out->data == in->data && out->poly_stride != in->poly_stride) return CKKS_EINVAL;
    size_t need = rescale_ws_bytes(C, (int)in->n_polys, (int)in->level, (int)mu, 1);
    if (!workspace || ws_bytes < need) return CKKS_ENOMEM;
    cudaSetDevice(C.device);
    cudaError_t err;
    double scale = in->scale;
    for (uint32_t j = 0; j < mu; ++j) scale /= (double)C.primes[in->level - 1 - j];
    uint32_t np = in->n_polys;
    int rc = run_rescale_ws(C, 1, (int)np, (int)in->level, (int)mu, tview(*in, C.N), tview(*out, C.N), workspace,
                            ws_bytes, S(stream), err);
    if (err != cudaSuccess || rc != 0) return cuda_fail(ctx, err == cudaSuccess ? cudaErrorUnknown : err);
    out->n_polys = np;
    out->level = ol;
    out->ntt_form = 1;
    out->scale = scale;
    return CKKS_OK;
}

int ckks_rescale(ckks_context *ctx, const ckks_tuple *in, ckks_tuple *out, void *workspace, size_t ws_bytes,
                 void *stream) {
    return ckks_rescale_multi(ctx, in, 1, out, workspace, ws_bytes, stream);
}

static int transform_api(ckks_context *ctx, const ckks_tuple *in, ckks_tuple *out, void *stream, bool fwd) {
    if (!ctx || !in || !out || !out->data) return CKKS_EINVAL;
    const Context &C = ctx->c;
    // plain transforms take any number of polynomials
    if (!in->data || in->level < 1 || in->level > (uint32_t)C.L || in->poly_stride < in->level || in->n_polys < 1 ||
        in->n_polys > 65535)
        return CKKS_EINVAL;
    if (out->poly_stride == 0) out->poly_stride = in->poly_stride;
    if (out->poly_stride < in->level) return CKKS_EINVAL;
    cudaSetDevice(C.device);
    cudaError_t err = transform_plain(C, fwd, 1, (int)in->n_polys, (int)in->level, tview(*in, C.N),
                                      tview(*out, C.N), S(stream));
    if (err != cudaSuccess) return cuda_fail(ctx, err);
    out->n_polys = in->n_polys;
    out->level = in->level;
    out->ntt_form = fwd ? 1 : 0;
    out->scale = in->scale;
    return CKKS_OK;
}

int ckks_ntt(ckks_context *ctx, const ckks_tuple *in, ckks_tuple *out, void *stream) {
    return transform_api(ctx, in, out, stream, true);
}

int ckks_intt(ckks_context *ctx, const ckks_tuple *in, ckks_tuple *out, void *stream) {
    return transform_api(ctx, in, out, stream, false);
}

int ckks_counters(ckks_context *ctx, ckks_op_counters *out, int reset) {
    if (!ctx || !out) return CKKS_EINVAL;
    Context &C = ctx->c;
    out->limb_ntt = C.counters[OP_LIMB_NTT].load();
    out->limb_intt = C.counters[OP_LIMB_INTT].load();
    out->ntt_phase = C.counters[OP_NTT_PHASE].load();
    out->intt_phase = C.counters[OP_INTT_PHASE].load();
    out->bconv = C.counters[OP_BCONV].load();
    out->kernels = C.counters[OP_KERNELS].load();
    if (reset)
        for (int i = 0; i < OP_COUNT; ++i) C.counters[i] = 0;
    return CKKS_OK;
}

static const char *kClassNames[KC_COUNT] = {"ntt_fwd_cols", "ntt_fwd_blocks", "ntt_inv_blocks", "ntt_inv_cols",
                                            "tensor",       "bconv",          "key_mac",        "rs_chain",
                                            "keys",         "automorphism"};

int ckks_profile_enable(ckks_context *ctx, int enable) {
    if (!ctx) return CKKS_EINVAL;
    Profiler &P = ctx->c.prof;
    if (enable) {
        P.recs.clear();
        P.used = 0;
    }
    P.on = enable != 0;
    return CKKS_OK;
}

int ckks_profile_read(ckks_context *ctx, ckks_kernel_stats *out, uint32_t max, uint32_t *n_out) {
    if (!ctx || !out || !n_out) return CKKS_EINVAL;
    cudaSetDevice(ctx->c.device);
    double ms[KC_COUNT] = {0}, by[KC_COUNT] = {0}, ops[KC_COUNT] = {0};
    uint64_t cnt[KC_COUNT] = {0};
    for (const ProfRec &r : ctx->c.prof.recs) {
        if (cudaEventSynchronize(r.b) != cudaSuccess) return CKKS_ECUDA;
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return CKKS_ECUDA;
        ms[r.cls] += t;
        by[r.cls] += r.bytes;
        ops[r.cls] += r.ops;
        cnt[r.cls] += 1;
    }
    uint32_t n = 0;
    for (int c = 0; c < KC_COUNT && n < max; ++c) {
        if (!cnt[c]) continue;
        memset(&out[n], 0, sizeof(out[n]));
        strncpy(out[n].name, kClassNames[c], sizeof(out[n].name) - 1);
        out[n].launches = cnt[c];
        out[n].total_ms = ms[c];
        out[n].alg_bytes = by[c];
        out[n].int_ops = ops[c];
        ++n;
    }
    *n_out = n;
    return CKKS_OK;
}

static int *tune_slot(ckks_context *ctx, const char *key, int &lo, int &hi) {
    if (!ctx || !key) return nullptr;
    if (!strcmp(key, "ntt_tile") || !strcmp(key, "ntt_tile_cols")) {
        lo = 1024;
        hi = 8192;
        return &ctx->c.tune_ntt_tile_cols;
    }
    if (!strcmp(key, "ntt_tile_blocks")) { lo = 1024; hi = 8192; return &ctx->c.tune_ntt_tile_blocks; }
    if (!strcmp(key, "bconv_threads")) { lo = 64; hi = 1024; return &ctx->c.tune_bconv_threads; }
    if (!strcmp(key, "mac_threads")) { lo = 64; hi = 1024; return &ctx->c.tune_mac_threads; }
    if (!strcmp(key, "inner_rescale")) { lo = 0; hi = 2; return &ctx->c.tune_inner_rescale; }
    if (!strcmp(key, "root_rescale")) { lo = 0; hi = 1; return &ctx->c.tune_root_rescale; }
    if (!strcmp(key, "moddown")) { lo = 0; hi = 1; return &ctx->c.tune_moddown; }
    if (!strcmp(key, "check_residues")) { lo = 0; hi = 1; return &ctx->c.tune_check_residues; }
    if (!strcmp(key, "nvtx")) { lo = 0; hi = 1; return &ctx->c.tune_nvtx; }
    if (!strcmp(key, "q1_forms")) { lo = 0; hi = 1; return &ctx->c.tune_q1; }
    if (!strcmp(key, "tensor_fixed")) { lo = 0; hi = 1; return &ctx->c.tune_tensor_fixed; }
    return nullptr;
}

int ckks_tune_set(ckks_context *ctx, const char *key, int value) {
    int lo, hi;
    int *slot = tune_slot(ctx, key, lo, hi);
    if (!slot || value < lo || value > hi) return CKKS_EINVAL;
    if (!strncmp(key, "ntt_tile", 8) && (value & (value - 1))) return CKKS_EINVAL;
    if ((!strcmp(key, "bconv_threads") || !strcmp(key, "mac_threads")) && value % 32) return CKKS_EINVAL;
    *slot = value;
    if (!strcmp(key, "ntt_tile")) ctx->c.tune_ntt_tile_blocks = value;  // both phases
    return CKKS_OK;
}

int ckks_tune_get(const ckks_context *ctx, const char *key, int *value) {
    int lo, hi;
    int *slot = tune_slot(const_cast<ckks_context *>(ctx), key, lo, hi);
    if (!slot || !value) return CKKS_EINVAL;
    *value = *slot;
    return CKKS_OK;
}

int ckks_check(ckks_context *ctx) {
    if (!ctx) return CKKS_EINVAL;
    if (ctx->c.sticky.load() != 0) return CKKS_ECUDA;
    cudaSetDevice(ctx->c.device);
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
        ctx->c.sticky.store((int)e);
        return CKKS_ECUDA;
    }
    return CKKS_OK;
}

const char *ckks_strerror(int code) {
    switch (code) {
    case CKKS_OK: return "ok";
    case CKKS_EINVAL: return "invalid argument";
    case CKKS_ELEVEL: return "level too low for the partition depth, or above L";
    case CKKS_EKEY: return "evaluation-key set lacks a needed ek_t";
    case CKKS_ENOMEM: return "workspace too small";
    case CKKS_ECUDA: return "CUDA error";
    case CKKS_ETIMEOUT: return "device wait timed out";
    case CKKS_EBUSY: return "admission refused";
    case CKKS_ECHECK: return "integrity check failed (a residue >= q, or the resident keys changed)";
    default: return "unknown error";
    }
}

}  // extern "C"
